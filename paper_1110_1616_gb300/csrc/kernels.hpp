// Launch interface between the C-ABI layer and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace amrk {

// Density and pressure floors (off when both are 0): a recovered density below
// rho is raised to rho before the velocity and pressure are formed, then a
// pressure below p is raised to p; every raise adds 1 to *events. They act on
// the primitives only (the stored conserved state is not changed), so where
// they act the advance is not conservative.
struct Floors {
  double rho = 0.0, p = 0.0;
  unsigned long long* events = nullptr;
};

// Per-patch descriptor in device memory.
struct DPatch {
  int lo[3], n[3], ext[3];
  int level;
  long long off;   // element offset of field 0 in a state buffer
  long long fs;    // elements per field array (padded)
  long long soff;  // element offset of the patch's scratch block
  long long boff;  // element offset of the patch's boundary capture block (fused 3D, levels > 0), or -1
};

// Scratch arrays per patch (each fs elements): W (8), Wh (8), S[d] (3x8),
// Ref (3), F[d] (3x8), E (3).
enum { SC_W = 0, SC_WH = 8, SC_S = 16, SC_REF = 40, SC_F = 43, SC_E = 67, SC_N = 70 };

struct LevelArgs {
  const DPatch* P;
  const int* ids;  // patch ids of this launch
  int npatch;
  int maxn[3];     // largest interior extent among them
  void* cur;       // state buffer read (base of all patches)
  void* nxt;       // state buffer written by the update
  void* scr;       // scratch base
  const double* dtp;
  double dtscale;  // dt = *dtp * dtscale
  double idx[3];   // 1/dx of this level
  double gamma;
  int w;           // extra ghost layers updated (0 or 2)
  int zlen;        // fused 3D advance: z planes per CTA (0: the whole column; -2: whole
                   // columns, those of the launch's last partial wave halved)
  int tail;        // set by the fused launcher: the last `tail` columns run as two halves
  // boundary capture buffer (fused 3D advance of a level > 0): the fluxes and
  // EMFs of every patch's boundary planes are written at P.boff; nullptr: none
  void* bnd;
  // direct halo reads (fused 3D advance of a level of equal patches tiling the
  // periodic domain, w = 0): per patch of the launch, the 27 patch ids of its
  // neighbours at (dx, dy, dz) in {-1, 0, 1}^3, index (dx+1) + 3 (dy+1) +
  // 9 (dz+1) (the patch itself at 13); the advance reads the cells and faces
  // of its halo from those patches' interiors instead of its own ghost cells,
  // so the level needs no same-level ghost fill. nullptr: read the ghosts.
  const int* nbr;
  Floors fl;
};

struct RowArgs {
  const DPatch* P;
  const int* rows;
  int64_t nrows;
  void* fbuf;        // buffer of the fine level (read)
  void* cbuf;        // buffer of the coarse level (written / read)
  void* scr;
  double* creg;      // coarse flux registers (row x 6)
  double* freg;      // fine flux registers (row x 2 x 6)
  double* ecreg;     // coarse EMF registers
  double* efreg;     // fine EMF registers (row x 2)
  const double* dtp;
  double dtscale;
  double idx[3];     // coarse level 1/dx
  double ratio[3][3];  // dx_n/dx_t on the coarse level
  int substep;       // 1 or 2
  double inflow[8];  // conserved inflow state (boundary fill)
  // regrid transfer: the old hierarchy's patch table and state buffer, and the
  // closure matrix (12 x 8)
  const DPatch* P2;
  const void* obuf;
  const double* K;
  // box copies: chunk table (box, first cell) per block
  const int* chunks;
  // same-level box copies: chunks [0, nsplit) are the cell boxes', the rest the
  // face boxes'; split_blocks = the blocks given to the cells (set at launch)
  int64_t nsplit;
  int split_blocks;
  // fine-side registers of the fused path: the boundary capture buffer the fine
  // level's advance wrote (nullptr: recompute the fluxes and EMFs)
  const void* bnd;
  Floors fl;  // the advance's floors (the register recompute repeats its recovery)
};

// Device work queue of the multi-level advance (k_advance_queue): one launch
// advances the levels whose sub-steps start together in the recursive order.
constexpr int QUEUE_MAX_LEVELS = 12;
constexpr unsigned ERR_QUEUE_TIMEOUT = 4u;  // error-word bit: a queue wait gave up
struct QueueLevel {
  LevelArgs a;          // the level's advance (buffers, dt, w, boundary capture)
  int ntx;              // tiles along x of the queue's tile variant for this level
  const int* boxes;     // same-level copy boxes of the sub-step (fill tasks)
  const int* chunks;    // their chunks (4 ints each)
};
struct QueueArgs {
  QueueLevel L[QUEUE_MAX_LEVELS];
  // tasks (4 ints): fill (code = slot << 4 | 1 | 2 for cell boxes, first
  // chunk, end chunk, destination patch id) or advance tile (code = slot << 4,
  // patch position in L[slot].a.ids, tile, patch id), in ticket order
  const int* tasks;
  int ntasks;
  const unsigned int* need;  // per patch id: fill tasks into it in this launch
  unsigned int* done;        // per patch id: fill tasks finished (zeroed before the launch)
  unsigned int* head;        // next ticket (zeroed before the launch)
  int* abort;                // set when a wait gave up (zeroed before the launch)
  unsigned int* err;         // the context's error word
  unsigned long long wait_ns;  // limit of one wait
};

struct CflArgs {
  const DPatch* P;
  const int* ids;
  int npatch;
  int maxn[3];
  const void* cur;
  double idx[3];
  double gamma;
  unsigned long long* slot;  // per-level max (bits of a non-negative double)
  unsigned int* err;
  Floors fl;
};

// sizes of a patch's boundary capture block (fused 3D path, levels > 0): the
// faces of its six boundary planes, and the tangential edges of those planes
__host__ __device__ __forceinline__ long long bnd_faces_total(const int* n) {
  return 2LL * ((long long)n[1] * n[2] + (long long)n[0] * n[2] + (long long)n[0] * n[1]);
}
__host__ __device__ __forceinline__ long long bnd_edges_total(const int* n) {
  long long t = 0;
  for (int e = 0; e < 3; ++e)
    for (int c = 0; c < 3; ++c)
      if (c != e) t += 2LL * n[c] * (n[3 - c - e] + 1);
  return t;
}

enum Variant { V_FP64 = 0, V_FP64_STRICT = 1, V_MIXED = 2 };

// positions per chunk of the box-list fill kernels (= threads per block of the
// prolongation and boundary kernels), and the ints of a same-level copy box
constexpr int FILL_CHUNK = 64;
constexpr int FILL_BOX_W = 16;

// A dense byte box over level cells (the regrid's clustering frame).
struct DenseBox {
  int off[3], n[3];
};

// the four row lists of a fine level's reflux and restriction (reflux cells,
// reflux faces, restriction cells, restriction faces) and, set by the
// launcher, the first block of each list's range
struct RRLists {
  const int* rows[4];
  long long n[4];
  unsigned b[5];
};

struct Ops {
  void (*advance)(const LevelArgs&, cudaStream_t, int* launches);
  void (*reg_coarse)(const RowArgs& faces, const RowArgs& edges, cudaStream_t, int* launches);
  void (*reg_fine)(const RowArgs& faces, const RowArgs& edges, cudaStream_t, int* launches);
  // ghost fill, all as boxes: rows = the box list, chunks of at most
  // FILL_CHUNK positions, nrows = the number of chunks. Same-level copies
  // (FILL_BOX_W-int boxes, cells and faces in one list; chunks (box, x0, q0,
  // nrows) of whole box rows), then prolongation and physical boundaries
  // (ghost boxes of amrmhd::GHOST_BOX_W ints; chunks (box, first position))
  void (*fill_runs)(const RowArgs&, cudaStream_t, int* launches);
  // the prolonged ghost cells and faces in one launch
  void (*prolong)(const RowArgs& cells, const RowArgs& faces, cudaStream_t, int* launches);
  void (*fill_bc_cells)(const RowArgs&, cudaStream_t, int* launches);
  void (*fill_bc_faces)(const RowArgs&, cudaStream_t, int* launches);
  // reflux (cells, faces) and restriction (cells, faces) of a fine level in
  // one launch: RowArgs gives the buffers and registers, RRLists the rows
  void (*reflux_restrict)(const RowArgs&, const RRLists&, cudaStream_t, int* launches);
  void (*cfl)(const CflArgs&, cudaStream_t, int* launches);
  // packed I/O of one field: to_state = 1 copies packed -> state
  void (*io)(const DPatch* P, const int* ids, int npatch, const int* maxn, void* state, double* packed,
             const long long* poff, int field, int to_state, cudaStream_t, int* launches);
  // the same for all 8 fields of a level in one launch: poff[kind] per field kind
  // (device array of 4 device pointers), foff[f] = field f's offset in packed;
  // packed holds doubles, or floats if packed_f32
  void (*io_all)(const DPatch* P, const int* ids, int npatch, const int* maxn, void* state, void* packed,
                 int packed_f32, const long long* const* poff, const long long* foff, int to_state, cudaStream_t,
                 int* launches);
  size_t elem;  // bytes per stored value
  // fused path (3D): one kernel per level advance, registers recomputed from the input state
  void (*prepare)();
  void (*advance_fused)(const LevelArgs&, int variant, cudaStream_t, int* launches);
  void (*reg_coarse_rc)(const RowArgs& faces, const RowArgs& edges, const double* idx, double gamma, cudaStream_t,
                        int* launches);
  void (*reg_fine_rc)(const RowArgs& faces, const RowArgs& edges, const double* idx, double gamma, cudaStream_t,
                      int* launches);
  // regrid: flagged cells of a level (global indices appended to out), the
  // transfer of a new fine level and its divergence-free closure
  void (*flag)(const LevelArgs&, double theta, int* out, unsigned long long* count, long long cap, cudaStream_t);
  void (*transfer_cells)(const RowArgs&, cudaStream_t, int* launches);
  void (*transfer_faces)(const RowArgs&, cudaStream_t, int* launches);
  void (*closure)(const RowArgs&, cudaStream_t, int* launches);
  // the multi-level queue advance (3D fused path); variant: 2 (16x8) or 3 (8x8)
  void (*advance_queue)(const QueueArgs&, int variant, cudaStream_t, int* launches);
  // regrid on the device: the level's cells (region) and its flagged cells
  // (flags) as bytes of the dense box of n[3] cells from off[3]
  void (*flag_dense)(const LevelArgs&, double theta, unsigned char* region, unsigned char* flags, DenseBox box,
                     cudaStream_t);
};

const Ops* ops_fast(int variant, int dim);    // V_FP64 and V_MIXED
const Ops* ops_strict(int dim);               // V_FP64_STRICT
void launch_fp_convert(long long n, const double* x, const float* y, float* xn, double* yw, float* xn_hw,
                       double* yw_hw, cudaStream_t s);
void launch_recover_mixed(long long n, const float* u, const float* bl, const float* br, double gm1, float* w,
                          cudaStream_t s);
void launch_fma_peak(int fp64, int blocks, int threads, int iters, void* out, cudaStream_t s);
void launch_grad_velocity(long long n, const double* u, const double* g, double* gv, cudaStream_t s);

void launch_set_scalar(double* p, double v, cudaStream_t s);
void launch_cfl_finalize(const unsigned long long* slots, int nlev, double cfl, double* dt_out, double* hist,
                         unsigned int* err, cudaStream_t s);
void launch_zero_u64(unsigned long long* p, int n, cudaStream_t s);

}  // namespace amrk
