// Uniform per-site interpreter for expression trees outside the compiled
// catalogue (FP64 storage).  The tree is flattened on the host into a short
// register program; every thread runs the same program on its own site, so
// control flow is uniform across the grid (no divergence), and the whole tree
// is still evaluated in one read/write pass (Sec. 3, Listing 1).  The register
// file lives in shared memory, laid out [register][real][thread] so that
// consecutive threads touch consecutive words; an instruction copies its
// operands into fixed-size arrays (their widths are known per operation), so
// the arithmetic runs on registers, and writes its result back.  The host
// sizes the shared memory to the registers the program uses: leaves are
// loaded at their first use and every register is freed after its last.
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
  int32_t nregs;   // registers the program uses (shared memory is sized to them)
  IIns ins[kIMax];
};

// The register file: real r of register g of this thread.
template <class M>
struct IRegs {
  typename M::R* base;
  int nt, tid;
  __device__ __forceinline__ typename M::R& at(int g, int r) const {
    return base[(g * 18 + r) * nt + tid];
  }
  template <int W>
  __device__ __forceinline__ void get(int g, typename M::R* v) const {
#pragma unroll
    for (int r = 0; r < W; ++r) v[r] = at(g, r);
  }
  template <int W>
  __device__ __forceinline__ void put(int g, const typename M::R* v) const {
#pragma unroll
    for (int r = 0; r < W; ++r) at(g, r) = v[r];
  }
};

// Object of W reals of field f (FP64 storage) at site s, link mu; g is the
// site's range guard (largest input high word, see dev_math.cuh).
template <class M, int W>
__device__ __forceinline__ void i_load(const FieldDesc& f, int64_t s, int mu, typename M::R* r,
                                       uint32_t& g) {
  const int64_t b = elem_base(f, s, mu);
  if constexpr (W == 1) {
    const uint2 v = ld8((const char*)f.ptr + b * 8);
    if constexpr (M::kGuard) g = guard_max(g, v.y, v.y);
    r[0] = M::from_bits(v.x, v.y);
  } else {
#pragma unroll
    for (int c = 0; c < W / 2; ++c) {
      const uint4 v = ld16((const char*)f.ptr + (b + c * f.s_c) * 16);
      if constexpr (M::kGuard) g = guard_max(g, v.y, v.w);
      split_complex<M>(v, r[2 * c], r[2 * c + 1]);
    }
  }
  M::template normalize_obj<W>(r);
}

template <class M, int W>
__device__ __forceinline__ void i_add(const IRegs<M>& R, const IIns& in, int sg) {
  typename M::R x[W], y[W], d[W];
  typename M::A acc[W];
  R.template get<W>(in.a, x);
  R.template get<W>(in.b, y);
#pragma unroll
  for (int r = 0; r < W; ++r) {
    M::template add<true, 1>(acc[r], x[r]);
    if (sg > 0) M::template add<false, 1>(acc[r], y[r]);
    else M::template add<false, -1>(acc[r], y[r]);
  }
  finish<M, W>(d, acc);
  R.template put<W>(in.dst, d);
}

template <class M, int W>
__device__ __forceinline__ void i_scale(const IRegs<M>& R, const IIns& in, const KParams& p) {
  typename M::R x[W], d[W];
  typename M::A acc[W];
  R.template get<W>(in.a, x);
  const typename M::R sc = M::scalar(p.sc[in.arg], p.sch[in.arg], p.scl[in.arg]);
#pragma unroll
  for (int r = 0; r < W; ++r) M::template fma<true, 1>(acc[r], sc, x[r]);
  finish<M, W>(d, acc);
  R.template put<W>(in.dst, d);
}

template <class M, int W>
__device__ __forceinline__ void i_store(const FieldDesc& dst, int64_t s, int mu, const IRegs<M>& R,
                                        int g) {
  typename M::R z[W];
  R.template get<W>(g, z);
  const int64_t b = elem_base(dst, s, mu);
  if constexpr (W == 1) {
    StoreReal::template store_acc<M>(dst.ptr, b, M::to_acc(z[0]));
  } else {
#pragma unroll
    for (int c = 0; c < W / 2; ++c) {
      typename M::A re[1] = {M::to_acc(z[2 * c])}, im[1] = {M::to_acc(z[2 * c + 1])};
      Store<P_F64>::template store_acc<M>(dst.ptr, b + c * dst.s_c, re, im);
    }
  }
}

// Run the program on site s into the register file R (g: range guard).
template <class M>
__device__ __forceinline__ void i_run(const KParams& p, const IProg& prog, const IRegs<M>& R,
                                      int64_t s, int mu, uint32_t& g) {
  using Rv = typename M::R;
  using Av = typename M::A;
  for (int pc = 0; pc < prog.n; ++pc) {
    const IIns in = prog.ins[pc];
    switch (in.op) {
      case I_LOAD: {
        Rv v[18];
        if (in.w == 18) {
          i_load<M, 18>(p.leaf[in.arg], s, mu, v, g);
          R.template put<18>(in.dst, v);
        } else if (in.w == 6) {
          i_load<M, 6>(p.leaf[in.arg], s, mu, v, g);
          R.template put<6>(in.dst, v);
        } else {
          i_load<M, 1>(p.leaf[in.arg], s, mu, v, g);
          R.template put<1>(in.dst, v);
        }
        break;
      }
      case I_MMUL: {
        Rv x[18], y[18], d[18];
        Av acc[18];
        R.template get<18>(in.a, x);
        R.template get<18>(in.b, y);
        mm_acc<M, true, 1, false, false>(acc, x, y);
        finish<M, 18>(d, acc);
        R.template put<18>(in.dst, d);
        break;
      }
      case I_MVMUL: {
        Rv x[18], y[6], d[6];
        Av acc[6];
        R.template get<18>(in.a, x);
        R.template get<6>(in.b, y);
        mv_acc<M, true, 1, false>(acc, x, y);
        finish<M, 6>(d, acc);
        R.template put<6>(in.dst, d);
        break;
      }
      case I_RMUL: {
        Rv x[1], y[1], d[1];
        Av acc[1];
        R.template get<1>(in.a, x);
        R.template get<1>(in.b, y);
        M::template fma<true, 1>(acc[0], x[0], y[0]);
        finish<M, 1>(d, acc);
        R.template put<1>(in.dst, d);
        break;
      }
      case I_ADD:
      case I_SUB: {
        const int sg = in.op == I_ADD ? 1 : -1;
        if (in.w == 18) i_add<M, 18>(R, in, sg);
        else if (in.w == 6) i_add<M, 6>(R, in, sg);
        else i_add<M, 1>(R, in, sg);
        break;
      }
      case I_SCALE: {
        if (in.w == 18) i_scale<M, 18>(R, in, p);
        else if (in.w == 6) i_scale<M, 6>(R, in, p);
        else i_scale<M, 1>(R, in, p);
        break;
      }
      default: {  // I_ADJ
        Rv x[18], t[18];
        R.template get<18>(in.a, x);
        adjoint<M>(t, x);
        R.template put<18>(in.dst, t);
        break;
      }
    }
  }
}

template <class M>
__device__ __forceinline__ void i_store_root(const KParams& p, const IProg& prog, const IRegs<M>& R,
                                             int64_t s, int mu) {
  if (prog.root_kind == KR) i_store<M, 1>(p.dst, s, mu, R, prog.root);
  else if (prog.root_kind == KV) i_store<M, 6>(p.dst, s, mu, R, prog.root);
  else i_store<M, 18>(p.dst, s, mu, R, prog.root);
}

// The range guard's path: the program again in native FP64 on this thread's
// slice of the register file (a double is no wider than any arithmetic's
// real, so it fits), then the store.  Out of line, off the hot loop.
__device__ __noinline__ void i_site_f64(const KParams& p, const IProg& prog, void* base, int nt,
                                        int tid, int64_t s, int mu) {
  const IRegs<MathF64> R{reinterpret_cast<double*>(base), nt, tid};
  uint32_t g = 0;
  i_run<MathF64>(p, prog, R, s, mu, g);
  i_store_root<MathF64>(p, prog, R, s, mu);
}

template <class M>
__global__ void __launch_bounds__(128) k_interp(const __grid_constant__ KParams p,
                                                const __grid_constant__ IProg prog) {
  using Rv = typename M::R;
  extern __shared__ __align__(16) unsigned char i_smem[];
  const IRegs<M> R{reinterpret_cast<Rv*>(i_smem), (int)blockDim.x, (int)threadIdx.x};
  const int mu = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < p.nvec; s += stride) {
    uint32_t g = p.gscal;
    i_run<M>(p, prog, R, s, mu, g);
    if (M::kGuard && g >= p.ghi) i_site_f64(p, prog, i_smem, (int)blockDim.x, (int)threadIdx.x, s, mu);
    else i_store_root<M>(p, prog, R, s, mu);
  }
}

// ------------------------------------------------------------------ host
namespace {
struct Builder {
  IProg prog;
  bool busy[kIRegs] = {};
  int leaf_reg[kMaxLeaves];
  int uses_left[kMaxLeaves] = {};  // leaf nodes of each slot not generated yet
  const Canon* c;
  int nscal = 0;
  int err = 0;

  int alloc() {
    for (int r = 0; r < kIRegs; ++r)
      if (!busy[r]) {
        busy[r] = true;
        if (r + 1 > prog.nregs) prog.nregs = r + 1;
        return r;
      }
    err = 1;
    return 0;
  }
  // free register r unless it holds a leaf that is still to be used
  void release(int r) {
    for (int l = 0; l < kMaxLeaves; ++l)
      if (leaf_reg[l] == r && uses_left[l] > 0) return;
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

  void count_uses(const su3s_expr* e) {
    if (e->op == 0) {
      ++uses_left[slot_of(e->f)];
      return;
    }
    if (e->a) count_uses(e->a);
    if (e->b) count_uses(e->b);
  }

  // returns the register holding the node's value
  int gen(const su3s_expr* e) {
    if (err) return 0;
    switch (e->op) {
      case 0: {  // a leaf: loaded at its first use
        const int l = slot_of(e->f);
        if (leaf_reg[l] < 0) {
          const int r = alloc();
          leaf_reg[l] = r;
          const int kind = e->f->kind;
          emit(IIns{I_LOAD, (int8_t)r, 0, (int8_t)kind, width(kind), (int8_t)l, {0, 0}});
        }
        --uses_left[l];
        return leaf_reg[l];
      }
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

template <class M>
cudaError_t launch_interp(const KParams& p, const IProg& prog, cudaStream_t st) {
  static_assert(!M::kGuard || sizeof(typename M::R) >= sizeof(double),
                "the range guard reruns the program in FP64 on the same register file");
  // shared memory: nregs registers of 18 reals per thread; 128 threads per
  // block while that fits in 200 KB, fewer for long programs
  const size_t per_thread = (size_t)prog.nregs * 18 * sizeof(typename M::R);
  int threads = 128;
  while (threads > 32 && per_thread * threads > (200u << 10)) threads /= 2;
  const size_t smem = per_thread * threads;
  const void* k = (const void*)&k_interp<M>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 1;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)per_sm * sm_count();               // one wave, grid-stride
  const int64_t need = (p.nvec + threads - 1) / threads;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  k_interp<M><<<dim3((unsigned)blocks, (unsigned)p.nmu), threads, smem, st>>>(p, prog);
  return cudaGetLastError();
}
}  // namespace

// Degree of a runtime tree (most factors in one term), as Degree<> of the
// compiled trees: it sets the range guard's bound.
static int degree(const su3s_expr* e) {
  switch (e->op) {
    case 0: return 1;
    case 1: return degree(e->a) + degree(e->b);
    case 4: return degree(e->a) + 1;
    case 5: return degree(e->a);
    default: {
      const int a = degree(e->a), b = degree(e->b);
      return a > b ? a : b;
    }
  }
}

int interp_eval(const su3s_expr* e, const Canon& c, su3s_field* dest, int math, cudaStream_t st) {
  Builder bld;
  memset(&bld.prog, 0, sizeof bld.prog);
  bld.c = &c;
  for (int l = 0; l < kMaxLeaves; ++l) bld.leaf_reg[l] = -1;
  bld.count_uses(e);
  int root = bld.gen(e);
  if (bld.err)
    return fail(SU3S_EUNSUPPORTED, "expression too large for the interpreter (%d registers, %d steps)",
                kIRegs, kIMax);
  bld.prog.root = root;
  bld.prog.root_kind = c.kind;
  KParams p;
  build_params(c, dest, 1, &p);
  p.ghi = guard_hi(degree(e));
  cudaError_t ce = math == MATH_F64  ? launch_interp<MathF64>(p, bld.prog, st)
                   : math == MATH_FX ? launch_interp<MathFX>(p, bld.prog, st)
                                     : launch_interp<MathDFScalar>(p, bld.prog, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "interpreter kernel launch");
  return SU3S_OK;
}

}  // namespace su3s
