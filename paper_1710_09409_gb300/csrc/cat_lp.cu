// Catalogue for reduced-precision storage (FP32 arithmetic) and two-row
// SU(3) storage.
#include "dev_kernels.cuh"
#include "internal.h"

namespace su3s {

template <int P>
static void lp_set() {
  using namespace cat;
  using M = MathF32;
  const int m = MATH_F32;
  reg_eval<MM, M, P>(m);
  reg_eval<AdjMM, M, P>(m);
  reg_eval<MAdjM, M, P>(m);
  reg_eval<MV, M, P>(m);
  reg_eval<E1, M, P>(m);
  reg_eval<CopyM, M, P>(m);
  reg_eval<CopyV, M, P>(m);
}

void register_cat_lp() {
  using namespace cat;
  lp_set<P_F32>();
  lp_set<P_BF16>();
  lp_set<P_F16>();
  // two-row storage: products and adjoints of SU(3) matrices only
  reg_eval<MM, MathF64, P_F64_C12>(MATH_F64);
  reg_eval<MM, MathDF, P_F64_C12>(MATH_DF);
  reg_eval<AdjMM, MathDF, P_F64_C12>(MATH_DF);
  reg_eval<MAdjM, MathDF, P_F64_C12>(MATH_DF);
  reg_eval<MMM, MathDF, P_F64_C12>(MATH_DF);
  reg_eval<CopyM, MathDF, P_F64_C12>(MATH_DF);
  reg_eval<MM, MathF32, P_F32_C12>(MATH_F32);
  reg_eval<AdjMM, MathF32, P_F32_C12>(MATH_F32);
  reg_eval<MAdjM, MathF32, P_F32_C12>(MATH_F32);
  reg_eval<CopyM, MathF32, P_F32_C12>(MATH_F32);
}

}  // namespace su3s
