// FP64 instantiation compiled without FMA contraction (--fmad=false): with the
// evaluation order of every formula fixed, this build reproduces a plain FP64
// CPU evaluation of the same formulas bit for bit.
#define AMRK_NS amrk_strict
#include "kernels_impl.cuh"

namespace amrk {

const Ops* ops_strict(int dim) {
  return dim == 3 ? amrk_strict::Impl<double, 3>::ops() : amrk_strict::Impl<double, 2>::ops();
}

}  // namespace amrk
