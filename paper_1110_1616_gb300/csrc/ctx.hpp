// Internal view of the library context, shared by the translation units of
// the C ABI (api.cu: forward path; adjoint.cu: discrete adjoint).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/amrmhd.h"
#include "hierarchy.hpp"
#include "kernels.hpp"

namespace amrapi {

struct DevList {  // a device int list with its row count
  int* p = nullptr;
  int64_t n = 0;
};

struct LevelDev {
  int* ids = nullptr;  // patch ids of the level (device)
  int npatch = 0;
  int maxn[3] = {1, 1, 1};
  // ghost fill of this level as boxes, each list with its chunks of at most
  // 64 positions: same-level copies (FILL_BOX_W ints per box, cells and faces
  // in one list, chunks of 4 ints: box, x0, q0, nrows), prolongation and
  // physical boundaries (GHOST_BOX_W ints per box, chunks of 2 ints: box,
  // first position)
  DevList runs, chunk_runs;
  int64_t runs_split = 0, runs2_split = 0;  // chunks of the cell boxes (listed first)
  DevList prol_cells, prol_faces, chunk_pcells, chunk_pfaces;
  DevList bc_cells, bc_faces, chunk_bcells, chunk_bfaces;
  // the same clipped to the ghosts within 2 cells of the interior (all that an
  // advance of the interior alone reads): used for sub-steps with w = 0
  DevList runs2, chunk_runs2;
  DevList bc_cells2, bc_faces2, chunk_bcells2, chunk_bfaces2;
  // one row per ghost position of the same fills (rows of amrmhd.h's ghost maps
  // split by kind), uploaded on demand for the adjoint's transposed fills
  DevList row_same_cells, row_same_faces, row_prol_cells, row_prol_faces, row_bc_cells, row_bc_faces;
  DevList cf_faces, cf_edges, emf_faces, restrict_cells, restrict_faces, reflux_cells;  // this level as fine level
  int64_t cf_face0 = 0, cf_edge0 = 0;  // global row offsets of this level's register rows
  // the 3D base level of a one-level hierarchy whose equal patches tile the
  // periodic domain: the fused advance reads its halo from the neighbour
  // patches (27 ids per patch, in the order of ids) and the level's same-level
  // fill is skipped
  DevList nbr;
  bool direct_halo = false;
  // host copies for the queue advance's fill tasks: per same-level copy record
  // (full and 2-cells-deep) its destination patch and its first chunk (one
  // more entry: the chunk count); has_bc: the level has physical-boundary boxes
  // (filled after its same-level copies, so its fill stays outside the queue)
  std::vector<int32_t> h_dst, h_dst2, h_chunk0, h_chunk0_2;
  bool has_bc = false;
};

// The queue advance's plan of one hierarchy: per batch k of a coarse step (the
// levels whose sub-steps start at finest sub-step k), its task list and the
// expected fill count per patch; counters shared by the batches.
struct QueuePlan {
  bool built = false;
  int variant = 3, withhold = 0, balance = 1;
  std::vector<double> batch_work;  // per batch: the cell updates of its advance tiles
  std::vector<int64_t> task_off;  // per batch: first task
  std::vector<int> task_n;        // per batch: task count
  std::vector<int> fill_in_queue; // per batch: 1 if the finest level's same-level fill is in the queue
  int* d_tasks = nullptr;         // 4 ints per task
  unsigned int* d_need = nullptr; // batch x npatch
  unsigned int* d_ctr = nullptr;  // done[npatch], head, abort
};

struct AdjWork;  // discrete-adjoint workspace (adjoint.cu)

}  // namespace amrapi

struct amrmhd_ctx {
  amrmhd_config cfg;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;  // created when the caller passes no stream
  std::string err;
  amrmhd::Hierarchy H;
  bool have_h = false, bound = false;
  // an intermediate regrid stage: ghost boxes only from level stage_ghost_from
  // on, no register maps and no advance scratch (it is filled, flagged and
  // copied, never advanced)
  bool stage_light = false;
  int stage_ghost_from = 0;
  int variant = amrk::V_FP64;
  const amrk::Ops* ops = nullptr;
  int64_t opt_advance = 0, opt_graph = 1, opt_tile = -1, opt_concurrent = 1, opt_host_io = 0, opt_direct_halo = 1;
  // the multi-level queue advance: on/off, its tile variant (2: 16x8, 3: 8x8),
  // and a test switch that withholds one fill signal (the wait times out)
  int64_t opt_queue = 0, opt_queue_tile = 3, opt_queue_withhold = 0, opt_queue_balance = 1;
  // z planes per CTA of the fused advance: -1 the autotuned length per level (else
  // the whole column), 0 the whole column, -2 whole columns with those of the
  // launch's last partial wave halved, n > 0 chunks of n planes
  int64_t opt_zchunk = -1;
  // density and pressure floors (0: off) and the device count of their raises
  double floor_rho = 0.0, floor_p = 0.0;
  unsigned long long* d_floor_events = nullptr;
  amrk::Floors floors() const {
    amrk::Floors f;
    if (floor_rho > 0.0 || floor_p > 0.0) {
      f.rho = floor_rho;
      f.p = floor_p;
      f.events = d_floor_events;
    }
    return f;
  }
  amrapi::QueuePlan qplan;
  // where the register, reflux and restriction maps are built: -1 on the device
  // when one is present, else on the host; 0 host; 1 device. Device-built lists
  // live in d_maps (list i at element dmap_off[i], dmap_n[i] rows); their host
  // copies in H are made on demand (dmaps_host) for the map export
  int64_t opt_device_maps = -1;
  bool dmaps = false, dmaps_host = false;
  int* d_maps = nullptr;
  int64_t dmap_off[6] = {0, 0, 0, 0, 0, 0}, dmap_n[6] = {0, 0, 0, 0, 0, 0};
  // the regrid's clustering: on the device (1, default) or the host (0), and
  // the device scratch of the device clustering (grown as needed)
  int64_t opt_device_cluster = 1;
  unsigned char* d_cluster = nullptr;
  size_t cluster_cap = 0;
  // autotuned fused tile per level, for the interior-only advance ([0]) and the
  // advance with 2 extended ghost layers ([1]) (-1: none)
  std::vector<std::array<int, 2>> tile_level;
  // autotuned z planes per CTA, same indexing (0: the whole column, -2: the
  // last partial wave's columns halved)
  std::vector<std::array<int, 2>> zlen_level;
  // the fused tile variant and z chunk of level l's advance with (wi = 1) or
  // without (wi = 0) the extended ghost layers, after options and autotuning
  int tile_of(int l, int wi) const {
    int v = opt_tile >= 0 ? (int)opt_tile : (variant == amrk::V_MIXED ? 2 : 3);
    if (opt_tile < 0 && (int)tile_level.size() > l && tile_level[l][wi] >= 0) v = tile_level[l][wi];
    return v;
  }
  int zlen_of(int l, int wi) const {
    if (opt_zchunk != -1) return (int)opt_zchunk;
    return (int)zlen_level.size() > l ? zlen_level[l][wi] : 0;
  }
  // the fused 3D kernel: forced (3), or by default (0) in mixed precision where it is
  // faster; FP64 defaults to the staged kernels (faster there: FP64-ALU bound)
  bool fused() const {
    return cfg.dim == 3 && (opt_advance == 3 || (opt_advance == 0 && cfg.precision == AMRMHD_MIXED));
  }
  // arena layout (bytes)
  std::vector<long long> off, fs, soff, boff;
  long long state_elems = 0, scr_elems = 0;
  size_t o_state[2] = {0, 0}, o_scr = 0, o_creg = 0, o_freg = 0, o_ecreg = 0, o_efreg = 0, o_stage = 0, o_bnd = 0;
  long long bnd_elems = 0;  // boundary capture blocks (fused 3D, levels > 0)
  size_t arena_bytes = 0;
  char* arena = nullptr;
  int64_t ncf = 0, nce = 0, stage_elems = 0;
  // packed I/O offsets: kind 0 cells, 1..3 faces along x,y,z
  std::vector<long long> poff[4];
  long long ptotal[4] = {0, 0, 0, 0};
  // library-owned device memory
  std::vector<void*> dev_allocs;
  amrk::DPatch* dP = nullptr;
  int* d_iota = nullptr;
  long long* d_poff[4] = {nullptr, nullptr, nullptr, nullptr};
  const long long** d_poff_tab = nullptr;  // device copy of d_poff (the 4 pointers)
  double* d_scal = nullptr;              // [0] CFL dt0, [1 + l] dt given to advance_level(l)
  unsigned long long* d_slots = nullptr;  // per-level CFL maxima + step counter
  unsigned int* d_err = nullptr;
  double* d_hist = nullptr;
  double* d_stage_all = nullptr;  // staging of the whole packed state (lazy)
  int64_t hist_cap = 0;
  std::vector<amrapi::LevelDev> lev;
  std::vector<int> cur, start;
  int maxn_all[3] = {1, 1, 1};
  // graphs, one per parity of level 0's buffer
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  std::vector<int> g_cur_before[2], g_cur_after[2], g_start_after[2];
  int g_launches[2] = {0, 0};
  long long launches = 0;
  // host wall time of the last regrid, microseconds: flagging, clustering,
  // hierarchy and map building with the stage arenas, data transfer
  long long regrid_us[6] = {0, 0, 0, 0, 0, 0};  // the five above, then the transfer maps
  long long maps_us[3] = {0, 0, 0};  // the last set_hierarchy: host build, ghost boxes, register maps
  // inter-level concurrency: side stream and fork/join events per level
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev_fork, ev_join;
  // the coarse step's CFL reduction beside the level-0 ghost fill
  cudaStream_t cfl_stream = nullptr;
  cudaEvent_t ev_cfl_fork = nullptr, ev_cfl_join = nullptr;
  // called after every ghost fill of op_level_step (level, sub-step): the
  // adjoint records the filled states there
  void (*after_fill)(amrmhd_ctx*, int, int) = nullptr;
  amrapi::AdjWork* adj = nullptr;
  // counts the calls that change the state: a recorded forward stays valid
  // for amrmhd_backward_recorded while the count is unchanged
  unsigned long long state_version = 0;
};

namespace amrapi {

amrmhd_status fail(amrmhd_ctx* c, amrmhd_status s, const std::string& m);
size_t align256(size_t x);
void* state_buf(amrmhd_ctx* ctx, int b);
amrk::LevelArgs level_args(amrmhd_ctx* ctx, int l, const double* dtp, double dtscale, int w);
amrk::RowArgs row_args(amrmhd_ctx* ctx, const DevList& L, int coarse_level);
void offset_regs(amrmhd_ctx* ctx, amrk::RowArgs& a, int l);
void level_idx(amrmhd_ctx* ctx, int l, double* idx);
void op_fill(amrmhd_ctx* ctx, int l, int s, int* nl);
void op_fill_same(amrmhd_ctx* ctx, int l, int s, int* nl);
void op_fill_rest(amrmhd_ctx* ctx, int l, int s, int* nl);
void op_level_registers(amrmhd_ctx* ctx, int l, const double* dtp, double dtscale, int s, void* bnd, int* nl);
void op_advance(amrmhd_ctx* ctx, int l, const double* dtp, double dtscale, int s, int* nl);
void op_reflux_restrict(amrmhd_ctx* ctx, int l, int* nl);
void op_level_step(amrmhd_ctx* ctx, int l, int s, int* nl, bool filled = false);
amrmhd_status check_bound(amrmhd_ctx* ctx);
amrmhd_status upload_fill_rows(amrmhd_ctx* ctx);
void adj_free(amrmhd_ctx* ctx);  // adjoint.cu
amrmhd_status device_register_maps(amrmhd_ctx* ctx);    // maps_dev.cu
amrmhd_status download_register_maps(amrmhd_ctx* ctx);  // maps_dev.cu
amrmhd_status device_ghost_boxes(amrmhd_ctx* ctx);      // maps_dev.cu
amrmhd_status device_transfer_maps(amrmhd_ctx* ctx, const amrmhd::Hierarchy& Hn, const amrmhd::Hierarchy& Ho, int lf,
                                   cudaStream_t st, std::vector<int32_t>& cells, std::vector<int32_t>& faces,
                                   std::vector<int32_t>& closure);  // maps_dev.cu
amrmhd_status cluster_level_device(amrmhd_ctx* ctx, amrmhd_ctx* c, int l, double theta,
                                   std::vector<std::array<int, 7>>& boxes);  // regrid_dev.cu

}  // namespace amrapi
