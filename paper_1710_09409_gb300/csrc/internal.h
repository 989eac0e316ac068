// Host-side internal declarations of the su3s library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/su3s.h"
#include "kparams.h"

#define SU3S_EXPORT extern "C" __attribute__((visibility("default")))

struct su3s_lattice {
  int L[4];
  int64_t V;
};

struct su3s_field {
  int L[4];
  int64_t V;      // real sites
  int64_t Vpad;   // padded sites
  int kind, nmu, prec, layout, block, ncomp;
  int elem_bytes;  // bytes of one stored complex (one real for real fields)
  void* ptr;
  size_t bytes;
  su3s::FieldDesc desc;
  CUtensorMap tmap;   // rows of 32-site tiles for the staged kernels (FP64 complex fields)
  bool tmap_ok;       // tmap was encoded
};

struct su3s_expr {
  std::atomic<int> ref{1};
  int op;     // 0 leaf, 1 mul, 2 add, 3 sub, 4 scale, 5 adj
  int kind;   // SU3S_MATRIX / VECTOR / REAL
  const su3s_expr* a = nullptr;
  const su3s_expr* b = nullptr;
  su3s_field* f = nullptr;
  double s = 0.0;
};

namespace su3s {

// error reporting (thread-local message)
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// canonical form of a runtime tree
struct Canon {
  std::string sig;
  std::vector<su3s_field*> leaves;  // by slot
  std::vector<double> scalars;      // by factor number
  int kind;
};
int canonicalize(const su3s_expr* e, Canon* out);

// field helpers
int check_same_shape(const su3s_field* a, const su3s_field* b, bool same_prec);
int sm_count();

// kernel registry
// Variants: 0 plain loads, 1 TMA-staged whole tile, 2 TMA-staged per leaf,
// 3 TMA-staged ring, 4 TMA-staged two tiles with two sites per lane.
constexpr int kNumVariants = 5;
struct EvalEntry {
  cudaError_t (*fn[kNumVariants])(const void*, dim3, dim3, cudaStream_t);
  const void* kernel[kNumVariants];
  int warp_bytes[kNumVariants];  // shared memory per warp of the staged variants
  int vps;
  int default_variant;           // chosen when no geometry is set
  int default_threads;           // 0: 128 staged / 256 plain
  int default_bps;               // blocks per SM, 0: occupancy / full grid
};

// A resolved launch: which variant, and its geometry.
struct Launch {
  cudaError_t (*fn)(const void*, dim3, dim3, cudaStream_t);
  dim3 grid, block;
  int variant;
};

const EvalEntry* find_eval(const std::string& sig, int prec, int math);
const EvalEntry* find_adjoint(const std::string& sig, int math);
void ensure_registered();

// launch geometry (tuned or default) for a kernel over nvec site vectors
void launch_geometry(const void* kernel, int64_t nvec, int nmu, dim3* grid, dim3* block);
void plain_geometry(int threads, int bps, int64_t nvec, int nmu, dim3* grid, dim3* block);
void set_geometry(const void* kernel, int64_t nvec, int nmu, int threads, int blocks_per_sm,
                  int variant = -1);
// resolve variant + geometry for an entry; tma_ok: the fields allow 32-site tiles
int plan_launch(const EvalEntry* e, int64_t nvec, int nmu, bool tma_ok, Launch* out);
bool tma_layout_ok(const su3s_field* f);
bool tma_tree_ok(const Canon& c, const su3s_field* dest);

// fill a KParams from a canonical tree and destination
int build_params(const Canon& c, const su3s_field* dest, int vps, KParams* p);

// arithmetic resolution for a storage precision
bool valid_math(int math);
int resolve_math(int prec, int math);

// interpreter
int interp_eval(const su3s_expr* e, const Canon& c, su3s_field* dest, int math, cudaStream_t st);

// pack / unpack kernels
cudaError_t launch_pack(const su3s_field* f, const double* canon, cudaStream_t st);
cudaError_t launch_unpack(const su3s_field* f, double* canon, cudaStream_t st);
cudaError_t launch_put_stored(const su3s_field* f, const void* src, cudaStream_t st);
cudaError_t launch_get_stored(const su3s_field* f, void* dst, cudaStream_t st);

// look up the static staging array of the no-allocation download on the
// current device (noalloc.cu); returns a status, cached per device
int prepare_static_stage();

// stream-ordered scratch from the library's memory pool
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st);
cudaError_t scratch_free(void* p, cudaStream_t st);

// catalogue registration (one per translation unit)
void register_cat_f64();
void register_cat_df();
void register_cat_df2();
void register_cat_lp();
void register_adj_f64();
void register_adj_df();
void register_cat_fx();
void register_cat_fx2();
void register_adj_fx();

}  // namespace su3s
