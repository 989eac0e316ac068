// Reverse-mode kernels, native FP64 arithmetic.
#include "dev_kernels.cuh"
#include "internal.h"

namespace su3s {

template <class M>
static void adj_set(int m) {
  using namespace cat;
  reg_adjoint<MM, M>(m);
  reg_adjoint<ScaleMM, M>(m);  // a scaled half of a split sum of two products
  reg_adjoint<AdjMM, M>(m);
  reg_adjoint<MAdjM, M>(m);
  reg_adjoint<MV, M>(m);
  reg_adjoint<E1, M>(m);
  reg_adjoint<E1Sub, M>(m);
  reg_adjoint<E1Lin, M>(m);
  reg_adjoint<E2, M>(m);
  reg_adjoint<MMM, M>(m);
  reg_adjoint<E3, M>(m);
  reg_adjoint<AddM, M>(m);
  reg_adjoint<ScaleM, M>(m);
  reg_adjoint<AdjM, M>(m);
  reg_adjoint<AddR, M>(m);
  reg_adjoint<MulR, M>(m);
  reg_adjoint<L2R, M>(m);
}

void register_adj_f64() { adj_set<MathF64>(MATH_F64); }

}  // namespace su3s
