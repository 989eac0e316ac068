// Reverse-mode kernels, pair-of-FP32 arithmetic.
#include "dev_kernels.cuh"
#include "internal.h"

namespace su3s {

// M: arithmetic of the single products; MS: the same arithmetic for trees of
// several products, whose reverse mode holds more operands at once
template <class M, class MS>
static void adj_set(int m) {
  using namespace cat;
  reg_adjoint<MM, M>(m);
  reg_adjoint<ScaleMM, M>(m);  // a scaled half of a split sum of two products
  reg_adjoint<AdjMM, M>(m);
  reg_adjoint<MAdjM, M>(m);
  reg_adjoint<MV, M>(m);
  reg_adjoint<E1, MS>(m);
  reg_adjoint<E1Sub, MS>(m);
  reg_adjoint<E1Lin, MS>(m);
  reg_adjoint<E2, MS>(m);
  reg_adjoint<MMM, MS>(m);
  reg_adjoint<E3, MS>(m);
  reg_adjoint<AddM, M>(m);
  reg_adjoint<ScaleM, M>(m);
  reg_adjoint<AdjM, M>(m);
  reg_adjoint<AddR, M>(m);
  reg_adjoint<MulR, M>(m);
  reg_adjoint<L2R, M>(m);
}

void register_adj_df() { adj_set<MathDF, MathDFScalar>(MATH_DF); }

}  // namespace su3s
