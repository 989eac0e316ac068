// Uniform per-site interpreter for expression trees outside the compiled
// catalogue (FP64 storage).  The tree is flattened on the host into a short
// register program; every thread runs the same program on its own site, so
// control flow is uniform across the grid (no divergence), and the whole tree
// is still evaluated in one read/write pass (Sec. 3, Listing 1).  Registers
// live in per-thread local memory.
#include <string.h>

#include <vector>

#include "dev_kernels.cuh"
#include "internal.h"

namespace su3s {

constexpr int kIRegs = 12;
constexpr int kIMax = 48;

enum IOp : int8_t { I_LOAD = 0, I_MMUL = 1, I_MVMUL = 2, I_RMUL = 3, I_ADD = 4, I_SUB = 5, I_SCALE = 6, I_ADJ = 7 };

struct IIns {
  int8_t op, dst, a, b;
  int8_t w;    // width in reals of the result (18, 6, 1)
  int8_t arg;  // leaf slot (LOAD, with kind in b) / factor index (SCALE)
  int8_t pad[2];
};

struct IProg {
  int32_t n;
  int32_t root;
  int32_t root_kind;
  int32_t pad;
  IIns ins[kIMax];
};

template <class M>
__device__ __forceinline__ void i_load(const FieldDesc& f, int kind, int64_t s, int mu,
                                       typename M::R* r) {
  const int64_t b = elem_base(f, s, mu);
  if (kind == KR) {
    r[0] = StoreReal::template load<M>(f.ptr, b);
    M::template normalize_obj<1>(r);
    return;
  }
  const int nc = kind == KM ? 9 : 3;
  for (int c = 0; c < nc; ++c) {
    typename M::R re[1], im[1];
    Store<P_F64>::template load<M>(f.ptr, b + c * f.s_c, re, im);
    r[2 * c] = re[0];
    r[2 * c + 1] = im[0];
  }
  if (kind == KM) M::template normalize_obj<18>(r);
  else M::template normalize_obj<6>(r);
}

// Accumulators of an object of w reals -> register values.
template <class M>
__device__ __forceinline__ void i_finish(typename M::R* d, const typename M::A* acc, int w) {
  if constexpr (M::kScaled) {
    if (w == 18) M::template finish_obj<18>(d, acc);
    else if (w == 6) M::template finish_obj<6>(d, acc);
    else M::template finish_obj<1>(d, acc);
  } else {
    for (int r = 0; r < w; ++r) d[r] = M::finish(acc[r]);
  }
}

template <class M>
__global__ void __launch_bounds__(256) k_interp(const __grid_constant__ KParams p,
                                                const __grid_constant__ IProg prog) {
  using R = typename M::R;
  using A = typename M::A;
  const int mu = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  R reg[kIRegs][18];
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < p.nvec; s += stride) {
    for (int pc = 0; pc < prog.n; ++pc) {
      const IIns in = prog.ins[pc];
      R* d = reg[in.dst];
      const R* x = reg[in.a];
      const R* y = reg[in.b];
      A acc[18];
      switch (in.op) {
        case I_LOAD: i_load<M>(p.leaf[in.arg], in.b, s, mu, d); continue;
        case I_MMUL: mm_acc<M, true, 1, false, false>(acc, x, y); break;
        case I_MVMUL: mv_acc<M, true, 1, false>(acc, x, y); break;
        case I_RMUL: M::template fma<true, 1>(acc[0], x[0], y[0]); break;
        case I_ADD:
          for (int r = 0; r < in.w; ++r) {
            M::template add<true, 1>(acc[r], x[r]);
            M::template add<false, 1>(acc[r], y[r]);
          }
          break;
        case I_SUB:
          for (int r = 0; r < in.w; ++r) {
            M::template add<true, 1>(acc[r], x[r]);
            M::template add<false, -1>(acc[r], y[r]);
          }
          break;
        case I_SCALE: {
          const R sc = M::scalar(p.sc[in.arg], p.sch[in.arg], p.scl[in.arg]);
          for (int r = 0; r < in.w; ++r) M::template fma<true, 1>(acc[r], sc, x[r]);
          break;
        }
        default: {  // I_ADJ
          R t[18];
          adjoint<M>(t, x);
          for (int r = 0; r < 18; ++r) d[r] = t[r];
          continue;
        }
      }
      i_finish<M>(d, acc, in.w);
    }
    const R* z = reg[prog.root];
    const int64_t b = elem_base(p.dst, s, mu);
    if (prog.root_kind == KR) {
      StoreReal::template store_acc<M>(p.dst.ptr, b, M::to_acc(z[0]));
    } else {
      const int nc = prog.root_kind == KM ? 9 : 3;
      for (int c = 0; c < nc; ++c) {
        A re[1] = {M::to_acc(z[2 * c])}, im[1] = {M::to_acc(z[2 * c + 1])};
        Store<P_F64>::template store_acc<M>(p.dst.ptr, b + c * p.dst.s_c, re, im);
      }
    }
  }
}

// ------------------------------------------------------------------ host
namespace {
struct Builder {
  IProg prog;
  bool busy[kIRegs] = {};
  int leaf_reg[kMaxLeaves];
  const Canon* c;
  int nscal = 0;
  int err = 0;

  int alloc() {
    for (int r = 0; r < kIRegs; ++r)
      if (!busy[r]) {
        busy[r] = true;
        return r;
      }
    err = 1;
    return 0;
  }
  void release(int r) {
    for (int l = 0; l < kMaxLeaves; ++l)
      if (leaf_reg[l] == r) return;  // leaf registers stay live
    busy[r] = false;
  }
  void emit(IIns in) {
    if (prog.n >= kIMax) {
      err = 2;
      return;
    }
    prog.ins[prog.n++] = in;
  }
  static int8_t width(int kind) { return kind == SU3S_MATRIX ? 18 : kind == SU3S_VECTOR ? 6 : 1; }

  int slot_of(const su3s_field* f) {
    for (size_t i = 0; i < c->leaves.size(); ++i)
      if (c->leaves[i] == f) return (int)i;
    return 0;
  }

  // returns the register holding the node's value
  int gen(const su3s_expr* e) {
    if (err) return 0;
    switch (e->op) {
      case 0: return leaf_reg[slot_of(e->f)];
      case 4: {
        int k = nscal++;  // factors numbered in the canonical (pre-order) order
        int a = gen(e->a);
        int d = alloc();
        emit(IIns{I_SCALE, (int8_t)d, (int8_t)a, 0, width(e->kind), (int8_t)k, {0, 0}});
        release(a);
        return d;
      }
      case 5: {
        int a = gen(e->a);
        int d = alloc();
        emit(IIns{I_ADJ, (int8_t)d, (int8_t)a, 0, 18, 0, {0, 0}});
        release(a);
        return d;
      }
      default: {
        int a = gen(e->a);
        int b = gen(e->b);
        int d = alloc();
        int8_t op;
        if (e->op == 1) op = e->kind == SU3S_MATRIX ? I_MMUL : e->kind == SU3S_VECTOR ? I_MVMUL : I_RMUL;
        else op = e->op == 2 ? I_ADD : I_SUB;
        emit(IIns{op, (int8_t)d, (int8_t)a, (int8_t)b, width(e->kind), 0, {0, 0}});
        release(a);
        release(b);
        return d;
      }
    }
  }
};
}  // namespace

int interp_eval(const su3s_expr* e, const Canon& c, su3s_field* dest, int math, cudaStream_t st) {
  Builder bld;
  memset(&bld.prog, 0, sizeof bld.prog);
  bld.c = &c;
  for (int l = 0; l < kMaxLeaves; ++l) bld.leaf_reg[l] = -1;
  for (size_t i = 0; i < c.leaves.size(); ++i) {
    int r = bld.alloc();
    bld.leaf_reg[i] = r;
    int kind = c.leaves[i]->kind;
    bld.emit(IIns{I_LOAD, (int8_t)r, 0, (int8_t)kind, Builder::width(kind), (int8_t)i, {0, 0}});
  }
  int root = bld.gen(e);
  if (bld.err)
    return fail(SU3S_EUNSUPPORTED, "expression too large for the interpreter (%d registers, %d steps)",
                kIRegs, kIMax);
  bld.prog.root = root;
  bld.prog.root_kind = c.kind;
  KParams p;
  build_params(c, dest, 1, &p);
  const void* kern = math == MATH_F64  ? (const void*)&k_interp<MathF64>
                     : math == MATH_FX ? (const void*)&k_interp<MathFX>
                                       : (const void*)&k_interp<MathDF>;
  dim3 grid, block;
  launch_geometry(kern, p.nvec, p.nmu, &grid, &block);
  if (math == MATH_F64) k_interp<MathF64><<<grid, block, 0, st>>>(p, bld.prog);
  else if (math == MATH_FX) k_interp<MathFX><<<grid, block, 0, st>>>(p, bld.prog);
  else k_interp<MathDF><<<grid, block, 0, st>>>(p, bld.prog);
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return cuda_fail(ce, "interpreter kernel launch");
  return SU3S_OK;
}

}  // namespace su3s
