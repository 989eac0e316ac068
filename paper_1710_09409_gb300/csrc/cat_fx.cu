// Catalogue of compiled trees, FP64 storage, shared-exponent fixed-point arithmetic:
// products and matrix-vector forms.
#include "dev_kernels.cuh"
#include "internal.h"

namespace su3s {

void register_cat_fx() {
  using namespace cat;
  constexpr int P = P_F64;
  using M = MathFX;
  const int m = MATH_FX;
  reg_eval<MM, M, P>(m);
  reg_eval<AdjMM, M, P>(m);
  reg_eval<MAdjM, M, P>(m);
  reg_eval<AdjMAdjM, M, P>(m);
  reg_eval<Square, M, P>(m);
  reg_eval<MV, M, P>(m);
  reg_eval<AdjMV, M, P>(m);
  reg_eval<MMV, M, P>(m);
  reg_eval<CopyM, M, P>(m);
  reg_eval<AdjM, M, P>(m);
  reg_eval<ScaleM, M, P>(m);
  reg_eval<AddM, M, P>(m);
  reg_eval<SubM, M, P>(m);
  reg_eval<AxpyM, M, P>(m);
  reg_eval<CopyV, M, P>(m);
  reg_eval<ScaleV, M, P>(m);
  reg_eval<AddV, M, P>(m);
  reg_eval<SubV, M, P>(m);
  reg_eval<AxpyV, M, P>(m);
  reg_eval<CopyR, M, P>(m);
  reg_eval<AddR, M, P>(m);
  reg_eval<SubR, M, P>(m);
  reg_eval<MulR, M, P>(m);
  reg_eval<ScaleR, M, P>(m);
  reg_eval<L2R, M, P>(m);
  // two-row storage
  reg_eval<MM, M, P_F64_C12>(m);
  reg_eval<AdjMM, M, P_F64_C12>(m);
  reg_eval<MAdjM, M, P_F64_C12>(m);
  reg_eval<MMM, M, P_F64_C12>(m);
  reg_eval<CopyM, M, P_F64_C12>(m);
}

}  // namespace su3s
