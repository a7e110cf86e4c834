// Instantiations of the apply kernel in F64 arithmetic (see sg_arith.h).
#include "sg_apply_kernel.cuh"

namespace sg {

void* select_kernel_f64(int dim, int k, int n_t) {
#define SG_CASE(D, KK, T) \
  if (dim == D && k == KK && n_t == T) return reinterpret_cast<void*>(&sg_apply_chunk_kernel<F64, D, KK, T>);
  SG_CASE(2, 1, 1) SG_CASE(2, 1, 2) SG_CASE(2, 1, 3) SG_CASE(2, 1, 4)
  SG_CASE(2, 2, 1) SG_CASE(2, 2, 2) SG_CASE(2, 2, 3) SG_CASE(2, 2, 4)
  SG_CASE(2, 3, 1) SG_CASE(2, 3, 2) SG_CASE(2, 3, 3) SG_CASE(2, 3, 4)
  SG_CASE(3, 1, 1) SG_CASE(3, 1, 2) SG_CASE(3, 2, 1) SG_CASE(3, 2, 2)
#undef SG_CASE
  return nullptr;
}

}  // namespace sg

SG_BOUNDS_FETCH(bounds_fetch_apply_f64)
