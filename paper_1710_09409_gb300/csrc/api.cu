// C ABI of the su3s library: lattices, fields, expression trees, evaluation
// planning and dispatch, upload/download, tuning, adjoint.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "dev_kernels.cuh"
#include "internal.h"

using namespace su3s;

namespace su3s {

// Device error word: kernels whose bounded pipeline waits give up record a
// code here; su3s_device_error reads and clears it.
__device__ int su3s_device_error_flag = 0;

// Address of the error word on the current device: every device that loads
// the library has its own copy, looked up once per device (with that device
// current) and cached.  Null if the lookup fails.
static int* device_error_ptr() {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static int* ptrs[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, su3s_device_error_flag) == cudaSuccess) ptrs[dev] = (int*)p;
  }
  return ptrs[dev];
}

// -1: choose per launch (TMA-staged where the layout allows), 0: plain loads, 1: TMA-staged
static std::atomic<int> g_pipeline_pref{-1};

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SU3S_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

static int ok() {
  g_err.clear();
  return SU3S_OK;
}

// ---------------------------------------------------------------- registry
static std::mutex g_reg_mu;
static std::map<std::tuple<std::string, int, int>, EvalEntry>& eval_reg() {
  static std::map<std::tuple<std::string, int, int>, EvalEntry> m;
  return m;
}
static std::map<std::pair<std::string, int>, EvalEntry>& adj_reg() {
  static std::map<std::pair<std::string, int>, EvalEntry> m;
  return m;
}

static EvalEntry make_entry(const Variants& v, int vps) {
  EvalEntry e{};
  for (int i = 0; i < kNumVariants; ++i) {
    e.fn[i] = v.fn[i];
    e.kernel[i] = v.kernel[i];
    e.warp_bytes[i] = v.warp_bytes[i];
  }
  e.vps = vps;
  e.default_variant = v.fn[1] ? v.default_variant : 0;
  e.default_threads = v.default_threads;
  e.default_bps = v.default_bps;
  return e;
}

void register_eval(const std::string& sig, int prec, int math, const Variants& v, int vps) {
  eval_reg()[std::make_tuple(sig, prec, math)] = make_entry(v, vps);
}

void register_adjoint(const std::string& sig, int math, const Variants& v) {
  adj_reg()[std::make_pair(sig, math)] = make_entry(v, 1);
}

void ensure_registered() {
  static std::once_flag once;
  std::call_once(once, [] {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    register_cat_f64();
    register_cat_df();
    register_cat_df2();
    register_cat_lp();
    register_adj_f64();
    register_adj_df();
    register_cat_fx();
    register_cat_fx2();
    register_adj_fx();
  });
}

const EvalEntry* find_eval(const std::string& sig, int prec, int math) {
  ensure_registered();
  auto it = eval_reg().find(std::make_tuple(sig, prec, math));
  return it == eval_reg().end() ? nullptr : &it->second;
}

const EvalEntry* find_adjoint(const std::string& sig, int math) {
  ensure_registered();
  auto it = adj_reg().find(std::make_pair(sig, math));
  return it == adj_reg().end() ? nullptr : &it->second;
}

// --------------------------------------------------------------- geometry
int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

struct Geo {
  int threads, bps, variant;  // variant -1: automatic
};
static std::mutex g_geo_mu;
static std::map<std::tuple<const void*, int64_t, int>, Geo> g_geo;

void set_geometry(const void* kernel, int64_t nvec, int nmu, int threads, int bps, int variant) {
  std::lock_guard<std::mutex> lk(g_geo_mu);
  Geo g{threads, bps, variant};
  g_geo[std::make_tuple(kernel, nvec, nmu)] = g;
}

static bool find_geometry(const void* kernel, int64_t nvec, int nmu, Geo* g) {
  std::lock_guard<std::mutex> lk(g_geo_mu);
  auto it = g_geo.find(std::make_tuple(kernel, nvec, nmu));
  if (it == g_geo.end()) return false;
  *g = it->second;
  return true;
}

// Whether the staged kernels can read field f: 32 sites of a component
// contiguous, and (matrices, vectors) a tensor map.
bool tma_layout_ok(const su3s_field* f) {
  if (f->layout != SU3S_SOA && f->block < 32) return false;
  return f->kind == SU3S_REAL || f->tmap_ok;
}

// ... for every leaf of a canonical tree and the destination.
bool tma_tree_ok(const Canon& c, const su3s_field* dest) {
  bool ok = tma_layout_ok(dest);
  for (const su3s_field* f : c.leaves) ok = ok && tma_layout_ok(f);
  return ok;
}

// Occupancy of a staged kernel (blocks per SM), cached per (kernel, threads).
static int staged_occupancy(const void* kernel, int threads, int warp_bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_pair(kernel, threads);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int n = 0;
  const size_t smem = (size_t)(threads / 32) * warp_bytes;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       8 * warp_bytes < smem_optin() ? 8 * warp_bytes : smem_optin());
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1)
    n = 1;
  cache[key] = n;
  return n;
}

int plan_launch(const EvalEntry* e, int64_t nvec, int nmu, bool tma_ok, Launch* out) {
  const int pref = g_pipeline_pref.load(std::memory_order_relaxed);
  Geo g{0, 0, pref};
  const bool set = find_geometry(e->kernel[0], nvec, nmu, &g);
  if (!set) {
    // the tree's default launch; a pipeline preference overrides its variant
    g.threads = e->default_threads;
    g.bps = e->default_bps;
    if (pref >= 0 && pref != e->default_variant) {
      g.threads = 0;
      g.bps = 0;
    }
  }
  const bool can_stage = e->fn[1] && tma_ok && nvec % 32 == 0;
  int variant = g.variant;
  if (variant < 0 || variant >= kNumVariants || !e->fn[variant]) variant = e->default_variant;
  if (!can_stage) {
    variant = 0;
    if (!set) {  // a staged default does not fit plain loads: take the plain defaults
      g.threads = 0;
      g.bps = 0;
    }
  }
  if (variant > 0) {
    int threads = g.threads > 0 ? g.threads : 128;
    if ((variant == 2 || variant == 3) && threads > 128) threads = 128;  // per-leaf / ring: <= 4 warps
    // at most the warps whose buffers fit one block's shared memory
    while (threads > 32 && (threads / 32) * e->warp_bytes[variant] > smem_optin()) threads -= 32;
    const int occ = staged_occupancy(e->kernel[variant], threads, e->warp_bytes[variant]);
    const int per_sm = g.bps > 0 && g.bps < occ ? g.bps : occ;
    // warps take 32-site tiles, or units of two tiles (two sites per lane)
    const int64_t ntiles = variant == 4 ? (nvec / 32 + 1) / 2 : nvec / 32, wpb = threads / 32;
    int64_t nb = ((int64_t)per_sm * sm_count() + nmu - 1) / nmu;
    const int64_t need = (ntiles + wpb - 1) / wpb;
    if (nb > need) nb = need;
    if (nb < 1) nb = 1;
    out->fn = e->fn[variant];
    out->grid = dim3((unsigned)nb, (unsigned)nmu, 1);
    out->block = dim3((unsigned)threads, 1, 1);
    out->variant = variant;
    return SU3S_OK;
  }
  out->fn = e->fn[0];
  out->variant = 0;
  plain_geometry(g.threads, g.bps, nvec, nmu, &out->grid, &out->block);
  return SU3S_OK;
}

void launch_geometry(const void* kernel, int64_t nvec, int nmu, dim3* grid, dim3* block) {
  Geo g{256, 0, -1};
  find_geometry(kernel, nvec, nmu, &g);
  plain_geometry(g.threads, g.bps, nvec, nmu, grid, block);
}

// Plain-load grid: `threads` per block (0: 256); bps > 0 gives a grid-stride
// grid of bps blocks per SM, else one site vector per thread.
void plain_geometry(int threads, int bps, int64_t nvec, int nmu, dim3* grid, dim3* block) {
  Geo g{threads, bps, -1};
  if (g.threads <= 0) g.threads = 256;
  int64_t nb;
  if (g.bps > 0) {
    nb = (int64_t)g.bps * sm_count();
    int64_t need = (nvec + g.threads - 1) / g.threads;
    if (nb > need) nb = need;
  } else {
    nb = (nvec + g.threads - 1) / g.threads;
  }
  if (nb < 1) nb = 1;
  if (nb > 0x7FFFFFFF) nb = 0x7FFFFFFF;
  *grid = dim3((unsigned)nb, (unsigned)nmu, 1);
  *block = dim3((unsigned)g.threads, 1, 1);
}

// ------------------------------------------------------------- mem pool
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st) {
  static cudaMemPool_t pool = nullptr;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!pool) {
      int dev = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e != cudaSuccess) return e;
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&pool, &props);
      if (e != cudaSuccess) {
        pool = nullptr;
        return e;
      }
      uint64_t thr = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      // An allocation must never make its stream wait for another stream's
      // work (uploads and downloads on different streams overlap): no reuse
      // through dependencies the pool would insert itself.
      int no = 0;
      cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

cudaError_t scratch_free(void* p, cudaStream_t st) { return cudaFreeAsync(p, st); }

// ------------------------------------------------------------ field shape
int check_same_shape(const su3s_field* a, const su3s_field* b, bool same_prec) {
  for (int d = 0; d < 4; ++d)
    if (a->L[d] != b->L[d]) return fail(SU3S_ESHAPE, "fields live on different lattices");
  if (a->nmu != b->nmu) return fail(SU3S_ESHAPE, "fields have different link counts");
  if (a->layout != b->layout || (a->layout == SU3S_AOSOA && a->block != b->block))
    return fail(SU3S_ESHAPE, "fields have different device layouts");
  if (same_prec && a->prec != b->prec)
    return fail(SU3S_ESHAPE, "fields have different storage precisions");
  return SU3S_OK;
}

static int ncomp_of(int kind, int prec) {
  if (kind == SU3S_MATRIX) return (prec == SU3S_F64_C12 || prec == SU3S_F32_C12) ? 6 : 9;
  if (kind == SU3S_VECTOR) return 3;
  return 1;
}

static int elem_bytes_of(int kind, int prec) {
  if (kind == SU3S_REAL) return 8;
  switch (prec) {
    case SU3S_F64:
    case SU3S_F64_C12: return 16;
    case SU3S_F32:
    case SU3S_F32_C12: return 8;
    default: return 4;
  }
}

static int layout_check(const su3s_lattice* lat, int kind, int nmu, int prec, int layout,
                        int block) {
  if (!lat) return fail(SU3S_EINVAL, "null lattice");
  if (kind < SU3S_MATRIX || kind > SU3S_REAL) return fail(SU3S_EINVAL, "bad field kind %d", kind);
  if (nmu < 1 || nmu > 8) return fail(SU3S_EINVAL, "links per site must be 1..8, got %d", nmu);
  if (prec < SU3S_F64 || prec > SU3S_F32_C12) return fail(SU3S_EINVAL, "bad precision %d", prec);
  if (layout != SU3S_SOA && layout != SU3S_AOSOA) return fail(SU3S_EINVAL, "bad layout %d", layout);
  if (layout == SU3S_AOSOA && (block < 4 || block > 1024 || (block & (block - 1))))
    return fail(SU3S_EINVAL, "site block must be a power of two in 4..1024, got %d", block);
  if (kind == SU3S_REAL && prec != SU3S_F64)
    return fail(SU3S_EUNSUPPORTED, "real fields are stored in FP64 only");
  if (kind != SU3S_MATRIX && (prec == SU3S_F64_C12 || prec == SU3S_F32_C12))
    return fail(SU3S_EUNSUPPORTED, "two-row storage exists for matrices only");
  return SU3S_OK;
}

static int64_t vpad_of(int64_t V, int layout, int block) {
  int64_t q = layout == SU3S_SOA ? 64 : (block < 4 ? 4 : block);
  return (V + q - 1) / q * q;
}

static void fill_desc(su3s_field* f) {
  FieldDesc& d = f->desc;
  d.ptr = f->ptr;
  const int64_t nc = f->ncomp;
  if (f->layout == SU3S_SOA) {
    d.logB = 31;
    d.mask = 0x7FFFFFFFu;
    d.s_c = f->Vpad;
    d.s_mu = nc * f->Vpad;
    d.s_blk = 0;
    d.row_blk = 0;
    d.row_mu = (int32_t)nc;
  } else {
    int lb = 0;
    while ((1 << lb) < f->block) ++lb;
    d.logB = lb;
    d.mask = (uint32_t)(f->block - 1);
    d.s_c = f->block;
    d.s_mu = nc * f->block;
    d.s_blk = (int64_t)f->nmu * nc * f->block;
    d.row_blk = (int32_t)(f->nmu * nc);
    d.row_mu = (int32_t)nc;
  }
}

// ---------------------------------------------------------- tensor maps
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no
// link against the driver library); null when no driver is present.
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();  // clear the lookup's error
  });
  return fn;
}

// Tensor map of an FP64 matrix or vector field for the staged kernels: a 2-D
// tensor of rows of s_c complex elements (2 s_c doubles; s_c = Vpad in the SoA
// layout, the site block otherwise), rows s_c * 16 bytes apart; the box is
// one 32-site tile (64 doubles) of every component of one object.
static void encode_tmap(su3s_field* f) {
  f->tmap_ok = false;
  memset(&f->tmap, 0, sizeof f->tmap);
  if ((f->prec != SU3S_F64 && f->prec != SU3S_F64_C12) || f->kind == SU3S_REAL) return;
  if (f->layout == SU3S_AOSOA && f->block < 32) return;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return;
  const uint64_t w = (uint64_t)f->desc.s_c;
  const uint64_t rows = (uint64_t)f->Vpad * f->nmu * f->ncomp / w;
  // tensor-copy coordinates are signed 32-bit: column 2*site (box end 2*w-1)
  // and row; larger fields (SoA beyond 2^30 sites) use the plain-load kernels
  if (2 * w > (1ull << 31) || rows > (1ull << 31)) return;
  const cuuint64_t dims[2] = {2 * w, rows};
  const cuuint64_t strides[1] = {w * 16};
  const cuuint32_t box[2] = {64, (cuuint32_t)f->ncomp};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(&f->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, f->ptr, dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  f->tmap_ok = r == CUDA_SUCCESS;
}

// ------------------------------------------------------------- canonical
static int canon_rec(const su3s_expr* e, Canon* c) {
  switch (e->op) {
    case 0: {
      int slot = -1;
      for (size_t i = 0; i < c->leaves.size(); ++i)
        if (c->leaves[i] == e->f) slot = (int)i;
      if (slot < 0) {
        slot = (int)c->leaves.size();
        c->leaves.push_back(e->f);
      }
      const char* k = e->kind == SU3S_MATRIX ? "M" : e->kind == SU3S_VECTOR ? "V" : "R";
      c->sig += k + std::to_string(slot);
      return SU3S_OK;
    }
    case 1:
    case 2:
    case 3: {
      c->sig += e->op == 1 ? "mul(" : e->op == 2 ? "add(" : "sub(";
      int rc = canon_rec(e->a, c);
      if (rc) return rc;
      c->sig += ",";
      rc = canon_rec(e->b, c);
      if (rc) return rc;
      c->sig += ")";
      return SU3S_OK;
    }
    case 4: {
      int k = (int)c->scalars.size();
      c->scalars.push_back(e->s);
      c->sig += "scale(s" + std::to_string(k) + ",";
      int rc = canon_rec(e->a, c);
      if (rc) return rc;
      c->sig += ")";
      return SU3S_OK;
    }
    case 5: {
      c->sig += "adj(";
      int rc = canon_rec(e->a, c);
      if (rc) return rc;
      c->sig += ")";
      return SU3S_OK;
    }
  }
  return fail(SU3S_EINVAL, "corrupt expression node");
}

int canonicalize(const su3s_expr* e, Canon* out) {
  out->sig.clear();
  out->leaves.clear();
  out->scalars.clear();
  int rc = canon_rec(e, out);
  if (rc) return rc;
  out->kind = e->kind;
  if ((int)out->leaves.size() > kMaxLeaves)
    return fail(SU3S_EUNSUPPORTED, "expression has %zu distinct fields; at most %d",
                out->leaves.size(), kMaxLeaves);
  if ((int)out->scalars.size() > kMaxScalars)
    return fail(SU3S_EUNSUPPORTED, "expression has %zu real factors; at most %d",
                out->scalars.size(), kMaxScalars);
  return SU3S_OK;
}

static std::atomic<int> g_default_math{SU3S_MATH_DF32};

bool valid_math(int math) {
  return math == SU3S_MATH_DEFAULT || math == SU3S_MATH_F64 || math == SU3S_MATH_DF32 ||
         math == SU3S_MATH_FX;
}

// Internal arithmetic id for a storage precision and a requested SU3S_MATH_*.
int resolve_math(int prec, int math) {
  if (prec == SU3S_F64 || prec == SU3S_F64_C12) {
    int m = math == SU3S_MATH_DEFAULT ? g_default_math.load(std::memory_order_relaxed) : math;
    return m == SU3S_MATH_F64 ? MATH_F64 : m == SU3S_MATH_FX ? MATH_FX : MATH_DF;
  }
  return MATH_F32;
}

static int math_for(int prec, int math) { return resolve_math(prec, math); }

static void split_scalar(double s, float* h, float* l) {
  float hh = (float)s;
  *h = hh;
  *l = (float)(s - (double)hh);
}

int build_params(const Canon& c, const su3s_field* dest, int vps, KParams* p) {
  memset(p, 0, sizeof *p);
  for (size_t i = 0; i < c.leaves.size(); ++i) {
    p->leaf[i] = c.leaves[i]->desc;
    p->tm[i] = c.leaves[i]->tmap;
  }
  p->dst = dest->desc;
  for (size_t k = 0; k < c.scalars.size(); ++k) {
    p->sc[k] = c.scalars[k];
    split_scalar(c.scalars[k], &p->sch[k], &p->scl[k]);
    // the real factors are inputs of every site: they open its range guard
    uint64_t bits;
    memcpy(&bits, &c.scalars[k], sizeof bits);
    const uint32_t hi = (uint32_t)(bits >> 32) & 0x7FFFFFFFu;
    if (hi > p->gscal) p->gscal = hi;
  }
  p->nvec = dest->Vpad / vps;
  p->nmu = dest->nmu;
  p->err = device_error_ptr();
  return SU3S_OK;
}

// Trees made of products and adjoints of matrices only (closed in SU(3)).
static bool su3_closed(const su3s_expr* e) {
  if (e->op == 0) return e->kind == SU3S_MATRIX;
  if (e->op == 1) return su3_closed(e->a) && su3_closed(e->b);
  if (e->op == 5) return su3_closed(e->a);
  return false;
}

static int check_eval(su3s_field* dest, const su3s_expr* e, Canon* c) {
  if (!dest || !e) return fail(SU3S_EINVAL, "null destination or expression");
  int rc = canonicalize(e, c);
  if (rc) return rc;
  if (c->kind != dest->kind)
    return fail(SU3S_ETYPE, "destination kind %d differs from the expression's kind %d",
                dest->kind, c->kind);
  for (su3s_field* f : c->leaves) {
    rc = check_same_shape(f, dest, true);
    if (rc) return rc;
  }
  if ((dest->prec == SU3S_F64_C12 || dest->prec == SU3S_F32_C12) && !su3_closed(e))
    return fail(SU3S_EUNSUPPORTED,
                "two-row storage holds SU(3) matrices: only products and adjoints of "
                "matrices can be stored in it");
  return SU3S_OK;
}

static int do_eval(su3s_field* dest, const su3s_expr* e, int math, cudaStream_t st) {
  Canon c;
  int rc = check_eval(dest, e, &c);
  if (rc) return rc;
  const int m = math_for(dest->prec, math);
  const EvalEntry* ent = find_eval(c.sig, dest->prec, m);
  if (!ent) {
    if (dest->prec == SU3S_F64) return interp_eval(e, c, dest, m, st);
    return fail(SU3S_EUNSUPPORTED, "no compiled kernel for %s in storage precision %d",
                c.sig.c_str(), dest->prec);
  }
  KParams p;
  build_params(c, dest, ent->vps, &p);
  Launch L;
  plan_launch(ent, p.nvec, p.nmu, tma_tree_ok(c, dest), &L);
  cudaError_t ce = L.fn(&p, L.grid, L.block, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "evaluation kernel launch");
  return ok();
}

}  // namespace su3s

// =================================================================== C ABI
SU3S_EXPORT const char* su3s_last_error(void) { return g_err.c_str(); }

SU3S_EXPORT int su3s_version(void) { return 10100; }

SU3S_EXPORT int su3s_lattice_create(int lx, int ly, int lz, int lt, su3s_lattice** out) {
  if (!out) return fail(SU3S_EINVAL, "null output handle");
  *out = nullptr;
  if (lx < 1 || ly < 1 || lz < 1 || lt < 1)
    return fail(SU3S_EINVAL, "lattice extents must be >= 1 (got %d %d %d %d)", lx, ly, lz, lt);
  int64_t v = (int64_t)lx * ly * lz * lt;
  if (v >= (int64_t)1 << 31) return fail(SU3S_EINVAL, "lattice volume %lld >= 2^31", (long long)v);
  su3s_lattice* l = new (std::nothrow) su3s_lattice;
  if (!l) return fail(SU3S_ENOMEM, "out of host memory");
  l->L[0] = lx;
  l->L[1] = ly;
  l->L[2] = lz;
  l->L[3] = lt;
  l->V = v;
  *out = l;
  return ok();
}

SU3S_EXPORT int su3s_lattice_destroy(su3s_lattice* lat) {
  delete lat;
  return ok();
}

SU3S_EXPORT int su3s_lattice_volume(const su3s_lattice* lat, int64_t* out) {
  if (!lat || !out) return fail(SU3S_EINVAL, "null argument");
  *out = lat->V;
  return ok();
}

SU3S_EXPORT int su3s_field_bytes(const su3s_lattice* lat, int kind, int nmu, int prec, int layout,
                                 int block, size_t* bytes) {
  if (!bytes) return fail(SU3S_EINVAL, "null output");
  int rc = layout_check(lat, kind, nmu, prec, layout, block);
  if (rc) return rc;
  int64_t vp = vpad_of(lat->V, layout, block);
  *bytes = (size_t)vp * nmu * ncomp_of(kind, prec) * elem_bytes_of(kind, prec);
  return ok();
}

SU3S_EXPORT int su3s_field_wrap(const su3s_lattice* lat, int kind, int nmu, int prec, int layout,
                                int block, void* dev_ptr, size_t bytes, su3s_field** out) {
  if (!out) return fail(SU3S_EINVAL, "null output handle");
  *out = nullptr;
  size_t need = 0;
  int rc = su3s_field_bytes(lat, kind, nmu, prec, layout, block, &need);
  if (rc) return rc;
  if (!dev_ptr) return fail(SU3S_EINVAL, "null device pointer");
  if (((uintptr_t)dev_ptr) & 15) return fail(SU3S_EINVAL, "device pointer is not 16-byte aligned");
  if (bytes < need)
    return fail(SU3S_ESHAPE, "buffer of %zu bytes is smaller than the %zu the field needs", bytes,
                need);
  su3s_field* f = new (std::nothrow) su3s_field;
  if (!f) return fail(SU3S_ENOMEM, "out of host memory");
  memcpy(f->L, lat->L, sizeof f->L);
  f->V = lat->V;
  f->Vpad = vpad_of(lat->V, layout, block);
  f->kind = kind;
  f->nmu = nmu;
  f->prec = prec;
  f->layout = layout;
  f->block = layout == SU3S_AOSOA ? block : 0;
  f->ncomp = ncomp_of(kind, prec);
  f->elem_bytes = elem_bytes_of(kind, prec);
  f->ptr = dev_ptr;
  f->bytes = bytes;
  fill_desc(f);
  encode_tmap(f);
  // Field creation may allocate: resolve here, on the current device, the
  // static staging array of su3s_field_download_static (which loads the
  // module holding it), so that the download itself never has to.  A failure
  // is reported by that download, not here.
  prepare_static_stage();
  *out = f;
  return ok();
}

SU3S_EXPORT int su3s_field_destroy(su3s_field* f) {
  delete f;
  return ok();
}

static size_t canon_doubles(const su3s_field* f) {
  int w = f->kind == SU3S_MATRIX ? 18 : f->kind == SU3S_VECTOR ? 6 : 1;
  return (size_t)f->V * f->nmu * w;
}

SU3S_EXPORT int su3s_field_pack(su3s_field* f, const double* dev_canonical, void* stream) {
  if (!f || !dev_canonical) return fail(SU3S_EINVAL, "null argument");
  cudaError_t e = launch_pack(f, dev_canonical, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pack kernel");
  return ok();
}

SU3S_EXPORT int su3s_field_unpack(const su3s_field* f, double* dev_canonical, void* stream) {
  if (!f || !dev_canonical) return fail(SU3S_EINVAL, "null argument");
  cudaError_t e = launch_unpack(f, dev_canonical, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "unpack kernel");
  return ok();
}

SU3S_EXPORT int su3s_field_upload(su3s_field* f, const double* host, size_t n, void* stream) {
  if (!f || !host) return fail(SU3S_EINVAL, "null argument");
  if (n != canon_doubles(f))
    return fail(SU3S_ESHAPE, "host array has %zu doubles, the field needs %zu", n, canon_doubles(f));
  cudaStream_t st = (cudaStream_t)stream;
  void* stage = nullptr;
  cudaError_t e = scratch_alloc(&stage, n * sizeof(double), st);
  if (e != cudaSuccess) return fail(SU3S_ENOMEM, "staging allocation of %zu bytes failed: %s",
                                    n * sizeof(double), cudaGetErrorString(e));
  e = cudaMemcpyAsync(stage, host, n * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_pack(f, (const double*)stage, st);
  cudaError_t e2 = scratch_free(stage, st);
  if (e != cudaSuccess) return cuda_fail(e, "upload");
  if (e2 != cudaSuccess) return cuda_fail(e2, "upload staging release");
  return ok();
}

SU3S_EXPORT int su3s_field_download(const su3s_field* f, double* host, size_t n, void* stream) {
  if (!f || !host) return fail(SU3S_EINVAL, "null argument");
  if (n != canon_doubles(f))
    return fail(SU3S_ESHAPE, "host array has %zu doubles, the field holds %zu", n, canon_doubles(f));
  cudaStream_t st = (cudaStream_t)stream;
  void* stage = nullptr;
  cudaError_t e = scratch_alloc(&stage, n * sizeof(double), st);
  if (e != cudaSuccess) return fail(SU3S_ENOMEM, "staging allocation of %zu bytes failed: %s",
                                    n * sizeof(double), cudaGetErrorString(e));
  e = launch_unpack(f, (double*)stage, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, stage, n * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = scratch_free(stage, st);
  if (e != cudaSuccess) return cuda_fail(e, "download");
  if (e2 != cudaSuccess) return cuda_fail(e2, "download staging release");
  return ok();
}

static size_t stored_bytes(const su3s_field* f) {
  return (size_t)f->V * f->nmu * f->ncomp * f->elem_bytes;
}

SU3S_EXPORT int su3s_field_stored_bytes(const su3s_field* f, size_t* bytes) {
  if (!f || !bytes) return fail(SU3S_EINVAL, "null argument");
  *bytes = stored_bytes(f);
  return ok();
}

SU3S_EXPORT int su3s_field_upload_stored(su3s_field* f, const void* host, size_t nbytes, void* stream) {
  if (!f || !host) return fail(SU3S_EINVAL, "null argument");
  if (nbytes != stored_bytes(f))
    return fail(SU3S_ESHAPE, "host array has %zu bytes, the field stores %zu", nbytes, stored_bytes(f));
  cudaStream_t st = (cudaStream_t)stream;
  void* stage = nullptr;
  cudaError_t e = cudaSuccess;
  if (nbytes > 0) {
    e = scratch_alloc(&stage, nbytes, st);
    if (e != cudaSuccess) return fail(SU3S_ENOMEM, "staging allocation of %zu bytes failed: %s",
                                      nbytes, cudaGetErrorString(e));
    e = cudaMemcpyAsync(stage, host, nbytes, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = launch_put_stored(f, stage, st);
  cudaError_t e2 = stage ? scratch_free(stage, st) : cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(e, "stored upload");
  if (e2 != cudaSuccess) return cuda_fail(e2, "upload staging release");
  return ok();
}

SU3S_EXPORT int su3s_field_download_stored(const su3s_field* f, void* host, size_t nbytes,
                                           void* stream) {
  if (!f || !host) return fail(SU3S_EINVAL, "null argument");
  if (nbytes != stored_bytes(f))
    return fail(SU3S_ESHAPE, "host array has %zu bytes, the field stores %zu", nbytes, stored_bytes(f));
  if (nbytes == 0) return ok();
  cudaStream_t st = (cudaStream_t)stream;
  void* stage = nullptr;
  cudaError_t e = scratch_alloc(&stage, nbytes, st);
  if (e != cudaSuccess) return fail(SU3S_ENOMEM, "staging allocation of %zu bytes failed: %s",
                                    nbytes, cudaGetErrorString(e));
  e = launch_get_stored(f, stage, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, stage, nbytes, cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = scratch_free(stage, st);
  if (e != cudaSuccess) return cuda_fail(e, "stored download");
  if (e2 != cudaSuccess) return cuda_fail(e2, "download staging release");
  return ok();
}

// ----------------------------------------------------------- expressions
static int new_node(int op, int kind, const su3s_expr* a, const su3s_expr* b, su3s_field* f,
                    double s, su3s_expr** out) {
  su3s_expr* e = new (std::nothrow) su3s_expr;
  if (!e) return fail(SU3S_ENOMEM, "out of host memory");
  e->op = op;
  e->kind = kind;
  e->a = a;
  e->b = b;
  e->f = f;
  e->s = s;
  if (a) const_cast<su3s_expr*>(a)->ref.fetch_add(1);
  if (b) const_cast<su3s_expr*>(b)->ref.fetch_add(1);
  *out = e;
  return ok();
}

SU3S_EXPORT int su3s_expr_leaf(su3s_field* f, su3s_expr** out) {
  if (!f || !out) return fail(SU3S_EINVAL, "null argument");
  return new_node(0, f->kind, nullptr, nullptr, f, 0.0, out);
}

SU3S_EXPORT int su3s_expr_mul(const su3s_expr* x, const su3s_expr* y, su3s_expr** out) {
  if (!x || !y || !out) return fail(SU3S_EINVAL, "null argument");
  int k;
  if (x->kind == SU3S_MATRIX && y->kind == SU3S_MATRIX) k = SU3S_MATRIX;
  else if (x->kind == SU3S_MATRIX && y->kind == SU3S_VECTOR) k = SU3S_VECTOR;
  else if (x->kind == SU3S_REAL && y->kind == SU3S_REAL) k = SU3S_REAL;
  else return fail(SU3S_ETYPE, "product of kinds %d and %d is not defined", x->kind, y->kind);
  return new_node(1, k, x, y, nullptr, 0.0, out);
}

SU3S_EXPORT int su3s_expr_add(const su3s_expr* x, const su3s_expr* y, su3s_expr** out) {
  if (!x || !y || !out) return fail(SU3S_EINVAL, "null argument");
  if (x->kind != y->kind) return fail(SU3S_ETYPE, "sum of different kinds");
  return new_node(2, x->kind, x, y, nullptr, 0.0, out);
}

SU3S_EXPORT int su3s_expr_sub(const su3s_expr* x, const su3s_expr* y, su3s_expr** out) {
  if (!x || !y || !out) return fail(SU3S_EINVAL, "null argument");
  if (x->kind != y->kind) return fail(SU3S_ETYPE, "difference of different kinds");
  return new_node(3, x->kind, x, y, nullptr, 0.0, out);
}

SU3S_EXPORT int su3s_expr_scale(double s, const su3s_expr* x, su3s_expr** out) {
  if (!x || !out) return fail(SU3S_EINVAL, "null argument");
  return new_node(4, x->kind, x, nullptr, nullptr, s, out);
}

SU3S_EXPORT int su3s_expr_adj(const su3s_expr* x, su3s_expr** out) {
  if (!x || !out) return fail(SU3S_EINVAL, "null argument");
  if (x->kind != SU3S_MATRIX) return fail(SU3S_ETYPE, "adjoint of a non-matrix");
  return new_node(5, SU3S_MATRIX, x, nullptr, nullptr, 0.0, out);
}

SU3S_EXPORT int su3s_expr_free(su3s_expr* e) {
  // iterative release of a reference-counted DAG
  std::vector<const su3s_expr*> todo;
  if (e) todo.push_back(e);
  while (!todo.empty()) {
    su3s_expr* n = const_cast<su3s_expr*>(todo.back());
    todo.pop_back();
    if (n->ref.fetch_sub(1) == 1) {
      if (n->a) todo.push_back(n->a);
      if (n->b) todo.push_back(n->b);
      delete n;
    }
  }
  return ok();
}

SU3S_EXPORT int su3s_expr_signature(const su3s_expr* e, char* buf, size_t cap) {
  if (!e || !buf || cap == 0) return fail(SU3S_EINVAL, "null argument");
  Canon c;
  int rc = canonicalize(e, &c);
  if (rc && rc != SU3S_EUNSUPPORTED) return rc;
  snprintf(buf, cap, "%s", c.sig.c_str());
  return ok();
}

SU3S_EXPORT int su3s_expr_num_leaves(const su3s_expr* e, int* n) {
  if (!e || !n) return fail(SU3S_EINVAL, "null argument");
  Canon c;
  int rc = canonicalize(e, &c);
  if (rc) return rc;
  *n = (int)c.leaves.size();
  return ok();
}

// ------------------------------------------------------------- evaluation
SU3S_EXPORT int su3s_eval(su3s_field* dest, const su3s_expr* e, void* stream) {
  return do_eval(dest, e, SU3S_MATH_DEFAULT, (cudaStream_t)stream);
}

SU3S_EXPORT int su3s_eval_math(su3s_field* dest, const su3s_expr* e, int math, void* stream) {
  if (!valid_math(math)) return fail(SU3S_EINVAL, "bad arithmetic %d", math);
  return do_eval(dest, e, math, (cudaStream_t)stream);
}

SU3S_EXPORT int su3s_set_default_math(int math) {
  if (math == SU3S_MATH_DEFAULT || !valid_math(math))
    return fail(SU3S_EINVAL, "default arithmetic must be SU3S_MATH_F64, SU3S_MATH_DF32 or SU3S_MATH_FX");
  g_default_math.store(math, std::memory_order_relaxed);
  return ok();
}

SU3S_EXPORT int su3s_catalogue(char* buf, size_t cap) {
  if (!buf || cap == 0) return fail(SU3S_EINVAL, "null argument");
  ensure_registered();
  std::string out;
  static const char* pn[] = {"f64", "f32", "bf16", "f16", "f64_c12", "f32_c12"};
  static const char* mn[] = {"", "f64", "df32", "f32", "fx"};
  for (auto& kv : eval_reg()) {
    out += "eval " + std::get<0>(kv.first) + " " + pn[std::get<1>(kv.first)] + " " +
           mn[std::get<2>(kv.first)] + "\n";
  }
  for (auto& kv : adj_reg()) out += "adjoint " + kv.first.first + " f64 " + mn[kv.first.second] + "\n";
  snprintf(buf, cap, "%s", out.c_str());
  return ok();
}

SU3S_EXPORT int su3s_set_launch(const su3s_field* dest, const su3s_expr* e, int math, int threads,
                                int blocks_per_sm) {
  if (threads < 32 || threads > 256 || threads % 32)
    return fail(SU3S_EINVAL, "threads per block must be a multiple of 32 in 32..256");
  if (blocks_per_sm < 0 || blocks_per_sm > 64) return fail(SU3S_EINVAL, "bad blocks per SM");
  Canon c;
  int rc = check_eval(const_cast<su3s_field*>(dest), e, &c);
  if (rc) return rc;
  const EvalEntry* ent = find_eval(c.sig, dest->prec, math_for(dest->prec, math));
  if (!ent) return fail(SU3S_EUNSUPPORTED, "no compiled kernel for %s", c.sig.c_str());
  set_geometry(ent->kernel[0], dest->Vpad / ent->vps, dest->nmu, threads, blocks_per_sm,
               g_pipeline_pref.load(std::memory_order_relaxed));
  return ok();
}

// Time every (variant, threads, blocks/SM) candidate of one registry entry on
// the caller's fields and keep the fastest as the geometry of (kernel, shape).
static int tune_entry(const EvalEntry* ent, const void* params, int64_t nvec, int nmu, bool tma_ok,
                      cudaStream_t st, int* threads_out, int* bps_out, int* variant_out,
                      float* best_ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fail(SU3S_ECUDA, "event creation failed");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(SU3S_ECUDA, "event creation failed");
  }
  const int th_c[] = {64, 128, 256};
  const int bps_c[] = {0, 2, 4, 8};
  const bool tma = ent->fn[1] && tma_ok && nvec % 32 == 0;
  float best = 1e30f;
  int bt = 256, bb = 0, bv = 0;
  int rc = SU3S_OK;
  for (int var = 0; var < (tma ? kNumVariants : 1) && rc == SU3S_OK; ++var) {
    if (!ent->fn[var]) continue;
    for (int th : th_c) {
      if ((var == 2 || var == 3) && th > 128) continue;  // per-leaf / ring: at most 4 warps
      for (int bps : bps_c) {
        set_geometry(ent->kernel[0], nvec, nmu, th, bps, var);
        Launch L;
        plan_launch(ent, nvec, nmu, tma, &L);
        cudaError_t ce = L.fn(params, L.grid, L.block, st);  // warm-up
        float ms = 1e30f;
        for (int trial = 0; trial < 2 && ce == cudaSuccess; ++trial) {
          ce = cudaEventRecord(e0, st);
          for (int r = 0; r < 3 && ce == cudaSuccess; ++r) ce = L.fn(params, L.grid, L.block, st);
          if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
          if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
          float t = 0.f;
          if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
          if (ce == cudaSuccess && t / 3.f < ms) ms = t / 3.f;
        }
        if (ce != cudaSuccess) {
          rc = cuda_fail(ce, "tuning launch");
          break;
        }
        if (ms < best) {
          best = ms;
          bt = th;
          bb = bps;
          bv = L.variant;
        }
      }
      if (rc != SU3S_OK) break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SU3S_OK) return rc;
  set_geometry(ent->kernel[0], nvec, nmu, bt, bb, bv);
  if (threads_out) *threads_out = bt;
  if (variant_out) *variant_out = bv;
  if (bps_out) *bps_out = bb;
  if (best_ms) *best_ms = best;
  return ok();
}

SU3S_EXPORT int su3s_tune(su3s_field* dest, const su3s_expr* e, int math, void* stream,
                          int* threads_out, int* bps_out, int* variant_out, float* best_ms) {
  Canon c;
  int rc = check_eval(dest, e, &c);
  if (rc) return rc;
  if (!valid_math(math)) return fail(SU3S_EINVAL, "bad arithmetic %d", math);
  const int m = math_for(dest->prec, math);
  const EvalEntry* ent = find_eval(c.sig, dest->prec, m);
  if (!ent) return fail(SU3S_EUNSUPPORTED, "no compiled kernel for %s", c.sig.c_str());
  KParams p;
  build_params(c, dest, ent->vps, &p);
  return tune_entry(ent, &p, p.nvec, p.nmu, tma_tree_ok(c, dest), (cudaStream_t)stream,
                    threads_out, bps_out, variant_out, best_ms);
}

SU3S_EXPORT int su3s_set_pipeline(int mode) {
  if (mode < -1 || mode > 4) return fail(SU3S_EINVAL, "pipeline mode must be -1, 0, 1, 2, 3 or 4");
  g_pipeline_pref.store(mode, std::memory_order_relaxed);
  return ok();
}

SU3S_EXPORT int su3s_device_error(int* code, void* stream) {
  if (!code) return fail(SU3S_EINVAL, "null argument");
  int* dev = device_error_ptr();
  if (!dev) return fail(SU3S_ECUDA, "device error word unavailable");
  static const int zero = 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(code, dev, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dev, &zero, sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
  return ok();
}

// One warp waits on a staging barrier that nothing completes (no copy is
// issued and nothing arrives), with the pipelines' bounded wait cut to `polls`
// polls: the wait gives up, the kernel records the time-out code in the device
// error word as a pipeline would, writes the SM cycles the wait took, and
// returns.
__global__ void k_selftest_wait(int* err, uint32_t polls, long long* cycles) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncwarp();
  const long long t0 = clock64();
  const bool ok = __all_sync(0xffffffffu, mbar_wait_polls(&bar, 0, polls));
  const long long t1 = clock64();
  if (threadIdx.x == 0) {
    if (!ok && err) atomicExch(err, kErrTmaTimeout);
    *cycles = ok ? -1 : t1 - t0;
  }
}

SU3S_EXPORT int su3s_selftest_bounded_wait(uint32_t polls, int64_t* cycles, void* stream) {
  if (!cycles) return fail(SU3S_EINVAL, "null argument");
  if (polls < 1 || polls > (1u << 20)) return fail(SU3S_EINVAL, "polls must be 1..2^20");
  cudaStream_t st = (cudaStream_t)stream;
  void* d = nullptr;
  cudaError_t e = scratch_alloc(&d, sizeof(long long), st);
  if (e != cudaSuccess) return fail(SU3S_ENOMEM, "scratch: %s", cudaGetErrorString(e));
  k_selftest_wait<<<1, 32, 0, st>>>(device_error_ptr(), polls, (long long*)d);
  e = cudaGetLastError();
  long long c = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&c, d, sizeof c, cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = scratch_free(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-test");
  if (e2 != cudaSuccess) return cuda_fail(e2, "bounded-wait self-test scratch");
  *cycles = c;
  return ok();
}

// ---------------------------------------------------------------- adjoint
// Checks and kernel parameters of a reverse-mode evaluation.
static int prepare_adjoint(const su3s_expr* e, const su3s_field* gout, su3s_field* const* gleaves,
                           int nleaves, int math, GParams* p, const EvalEntry** ent, bool* tma) {
  if (!e || !gout) return fail(SU3S_EINVAL, "null argument");
  Canon c;
  int rc = canonicalize(e, &c);
  if (rc) return rc;
  if (nleaves != (int)c.leaves.size())
    return fail(SU3S_EINVAL, "expression has %zu distinct fields, %d gradients given",
                c.leaves.size(), nleaves);
  if (gout->kind != c.kind) return fail(SU3S_ETYPE, "gradient field kind differs from the tree's");
  if (gout->prec != SU3S_F64) return fail(SU3S_EUNSUPPORTED, "adjoint needs FP64 storage");
  for (size_t i = 0; i < c.leaves.size(); ++i) {
    rc = check_same_shape(c.leaves[i], gout, true);
    if (rc) return rc;
    if (gleaves && gleaves[i]) {
      rc = check_same_shape(gleaves[i], gout, true);
      if (rc) return rc;
      if (gleaves[i]->kind != c.leaves[i]->kind)
        return fail(SU3S_ETYPE, "gradient %zu has the wrong kind", i);
    }
  }
  // Gradients are written while leaves and dL/dZ are still being read (and a
  // site out of the FP64-accurate range reads them again): no overlap.
  const auto overlap = [](const su3s_field* a, const su3s_field* b) {
    const char* pa = (const char*)a->ptr;
    const char* pb = (const char*)b->ptr;
    return pa < pb + b->bytes && pb < pa + a->bytes;
  };
  for (size_t i = 0; gleaves && i < c.leaves.size(); ++i) {
    if (!gleaves[i]) continue;
    bool clash = overlap(gleaves[i], gout);
    for (size_t j = 0; j < c.leaves.size(); ++j) {
      clash = clash || overlap(gleaves[i], c.leaves[j]);
      if (j != i && gleaves[j]) clash = clash || overlap(gleaves[i], gleaves[j]);
    }
    if (clash)
      return fail(SU3S_EINVAL, "gradient %zu overlaps a leaf, dL/dZ or another gradient", i);
  }
  if (!valid_math(math)) return fail(SU3S_EINVAL, "bad arithmetic %d", math);
  const int m = math_for(SU3S_F64, math);
  *ent = find_adjoint(c.sig, m);
  if (!*ent) return fail(SU3S_EUNSUPPORTED, "no compiled adjoint kernel for %s", c.sig.c_str());
  memset(p, 0, sizeof *p);
  build_params(c, gout, 1, &p->k);
  p->gout = gout->desc;
  for (size_t i = 0; i < c.leaves.size(); ++i)
    if (gleaves && gleaves[i]) p->gleaf[i] = gleaves[i]->desc;
  p->tm_gout = gout->tmap;
  *tma = tma_tree_ok(c, gout);   // leaves and dL/dZ are staged; gradients are stored per site
  return SU3S_OK;
}

// Reverse mode of a sum or difference of two products of distinct leaves
// (a*b + c*d, a*b - c*d, s0 a*b + s1 c*d) as two single-product reverse-mode
// launches, (a, b, dL/dZ -> dA, dB) and (c, d, dL/dZ -> dC, dD).  Each launch
// reads dL/dZ, so the split moves one object more per site (1,440 instead of
// 1,296 B per site in FP64), but each kernel holds the operands of one
// product only.  su3s_tune_adjoint times both forms and keeps the faster.
struct SplitAdjoint {
  GParams p[2];
  const EvalEntry* ent[2];
  bool tma[2];
};

static bool plan_split_adjoint(const su3s_expr* e, const su3s_field* gout,
                               su3s_field* const* gleaves, int math, SplitAdjoint* out) {
  Canon c;
  if (canonicalize(e, &c) || c.leaves.size() != 4) return false;
  double s[2];
  if (c.sig == "add(mul(M0,M1),mul(M2,M3))") {
    s[0] = 1.0;
    s[1] = 1.0;
  } else if (c.sig == "sub(mul(M0,M1),mul(M2,M3))") {
    s[0] = 1.0;
    s[1] = -1.0;
  } else if (c.sig == "add(scale(s0,mul(M0,M1)),scale(s1,mul(M2,M3)))") {
    s[0] = c.scalars[0];
    s[1] = c.scalars[1];
  } else {
    return false;
  }
  const int m = math_for(SU3S_F64, math);
  for (int h = 0; h < 2; ++h) {
    Canon ch;
    ch.kind = SU3S_MATRIX;
    ch.leaves = {c.leaves[2 * h], c.leaves[2 * h + 1]};
    if (s[h] == 1.0) {
      ch.sig = "mul(M0,M1)";
    } else {
      ch.sig = "scale(s0,mul(M0,M1))";
      ch.scalars = {s[h]};
    }
    out->ent[h] = find_adjoint(ch.sig, m);
    if (!out->ent[h]) return false;
    GParams& p = out->p[h];
    memset(&p, 0, sizeof p);
    build_params(ch, gout, 1, &p.k);
    p.gout = gout->desc;
    p.tm_gout = gout->tmap;
    for (int i = 0; i < 2; ++i)
      if (gleaves && gleaves[2 * h + i]) p.gleaf[i] = gleaves[2 * h + i]->desc;
    out->tma[h] = tma_tree_ok(ch, gout);
  }
  return true;
}

// Whether the reverse mode of a tree, arithmetic and shape runs split (set by
// su3s_tune_adjoint; absent: kSplitDefault).
static std::mutex g_adj_mode_mu;
static std::map<std::tuple<std::string, int, int64_t, int>, bool>& adj_mode() {
  static std::map<std::tuple<std::string, int, int64_t, int>, bool> m;
  return m;
}
static constexpr bool kSplitDefault = true;

// -1: tuned choice (or kSplitDefault); 0: always fused; 1: always split
static std::atomic<int> g_split_pref{-1};

static bool use_split(const std::string& sig, int m, int64_t nvec, int nmu) {
  const int pref = g_split_pref.load(std::memory_order_relaxed);
  if (pref >= 0) return pref == 1;
  std::lock_guard<std::mutex> lk(g_adj_mode_mu);
  auto it = adj_mode().find(std::make_tuple(sig, m, nvec, nmu));
  return it == adj_mode().end() ? kSplitDefault : it->second;
}

static cudaError_t launch_planned(const EvalEntry* ent, const GParams& p, bool tma, cudaStream_t st) {
  Launch L;
  plan_launch(ent, p.k.nvec, p.k.nmu, tma, &L);
  return L.fn(&p, L.grid, L.block, st);
}

SU3S_EXPORT int su3s_set_adjoint_split(int mode) {
  if (mode < -1 || mode > 1) return fail(SU3S_EINVAL, "split mode must be -1, 0 or 1");
  g_split_pref.store(mode, std::memory_order_relaxed);
  return ok();
}

SU3S_EXPORT int su3s_eval_adjoint(const su3s_expr* e, const su3s_field* gout,
                                  su3s_field* const* gleaves, int nleaves, int math, void* stream) {
  GParams p;
  const EvalEntry* ent = nullptr;
  bool tma = false;
  int rc = prepare_adjoint(e, gout, gleaves, nleaves, math, &p, &ent, &tma);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Canon c;
  canonicalize(e, &c);
  SplitAdjoint sp;
  cudaError_t ce;
  if (use_split(c.sig, math_for(SU3S_F64, math), p.k.nvec, p.k.nmu) &&
      plan_split_adjoint(e, gout, gleaves, math, &sp)) {
    ce = launch_planned(sp.ent[0], sp.p[0], sp.tma[0], st);
    if (ce == cudaSuccess) ce = launch_planned(sp.ent[1], sp.p[1], sp.tma[1], st);
  } else {
    ce = launch_planned(ent, p, tma, st);
  }
  if (ce != cudaSuccess) return cuda_fail(ce, "adjoint kernel launch");
  return ok();
}

// Best of two runs of three launches of both halves of a split reverse mode.
static int time_split(const SplitAdjoint& sp, cudaStream_t st, float* ms_out) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fail(SU3S_ECUDA, "event creation failed");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(SU3S_ECUDA, "event creation failed");
  }
  float best = 1e30f;
  cudaError_t ce = cudaSuccess;
  for (int trial = 0; trial < 3 && ce == cudaSuccess; ++trial) {  // trial 0 warms up
    ce = cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && ce == cudaSuccess; ++r) {
      ce = launch_planned(sp.ent[0], sp.p[0], sp.tma[0], st);
      if (ce == cudaSuccess) ce = launch_planned(sp.ent[1], sp.p[1], sp.tma[1], st);
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float t = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
    if (ce == cudaSuccess && trial > 0 && t / 3.f < best) best = t / 3.f;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ce != cudaSuccess) return cuda_fail(ce, "timing the split reverse mode");
  *ms_out = best;
  return SU3S_OK;
}

SU3S_EXPORT int su3s_tune_adjoint(const su3s_expr* e, const su3s_field* gout,
                                  su3s_field* const* gleaves, int nleaves, int math, void* stream,
                                  int* threads_out, int* bps_out, int* variant_out,
                                  float* best_ms) {
  GParams p;
  const EvalEntry* ent = nullptr;
  bool tma = false;
  int rc = prepare_adjoint(e, gout, gleaves, nleaves, math, &p, &ent, &tma);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int th = 0, bps = 0, var = 0;
  float ms = 0.f;
  rc = tune_entry(ent, &p, p.k.nvec, p.k.nmu, tma, st, &th, &bps, &var, &ms);
  if (rc) return rc;
  Canon c;
  canonicalize(e, &c);
  const int m = math_for(SU3S_F64, math);
  SplitAdjoint sp;
  if (plan_split_adjoint(e, gout, gleaves, math, &sp)) {
    // tune each distinct half kernel, then time the pair as it runs
    int th2 = 0, bps2 = 0, var2 = 0;
    float ms_half = 0.f;
    rc = tune_entry(sp.ent[0], &sp.p[0], p.k.nvec, p.k.nmu, sp.tma[0], st, &th2, &bps2, &var2,
                    &ms_half);
    if (!rc && sp.ent[1] != sp.ent[0])
      rc = tune_entry(sp.ent[1], &sp.p[1], p.k.nvec, p.k.nmu, sp.tma[1], st, nullptr, nullptr,
                      nullptr, &ms_half);
    float ms_split = 0.f;
    if (!rc) rc = time_split(sp, st, &ms_split);
    if (rc) return rc;
    const bool split = ms_split < ms;
    {
      std::lock_guard<std::mutex> lk(g_adj_mode_mu);
      adj_mode()[std::make_tuple(c.sig, m, p.k.nvec, p.k.nmu)] = split;
    }
    if (split) {
      th = th2;
      bps = bps2;
      var = 10 + var2;
      ms = ms_split;
    }
  }
  if (threads_out) *threads_out = th;
  if (bps_out) *bps_out = bps;
  if (variant_out) *variant_out = var;
  if (best_ms) *best_ms = ms;
  return ok();
}
