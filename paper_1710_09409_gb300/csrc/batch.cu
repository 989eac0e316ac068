// Batched evaluation: many (destination, tree) items over lattices of uneven
// volumes run in one persistent kernel.  The host cuts every item into tiles
// of site vectors; a fixed grid of blocks (sized from occupancy) walks the
// tile list round-robin, and each tile dispatches on its item's tree (uniform
// within the block).  The launch, plus separate launches for items whose tree
// the persistent kernel does not cover, is captured once into a CUDA graph
// and replayed with a single cudaGraphLaunch.
#include <string.h>

#include <string>
#include <vector>

#include "dev_kernels.cuh"
#include "internal.h"

struct su3s_batch;

namespace su3s {

struct BItem {
  KParams k;
  int32_t tree;
  int32_t pad;
};

struct BTile {
  int32_t item;
  int32_t mu;
  int64_t t0, t1;
};

// Trees the persistent kernel covers (index = BItem::tree).
static const char* const kBatchTrees[] = {
    "mul(M0,M1)",                                         // 0
    "add(mul(M0,M1),mul(M2,M3))",                         // 1
    "mul(M0,V1)",                                         // 2
    "add(mul(mul(M0,M1),M2),scale(s0,M3))",               // 3
    "sub(mul(adj(M0),M1),mul(M1,adj(M0)))",               // 4
    "mul(mul(M0,M1),M2)",                                 // 5
    "add(scale(s0,mul(M0,M1)),scale(s1,mul(M2,M3)))",     // 6
    "mul(adj(M0),M1)",                                    // 7
};
constexpr int kNumBatchTrees = 8;

template <class M>
__global__ void __launch_bounds__(256) k_batch(const BItem* __restrict__ items,
                                               const BTile* __restrict__ tiles, int64_t ntiles) {
  for (int64_t i = blockIdx.x; i < ntiles; i += gridDim.x) {
    const BTile T = tiles[i];
    const BItem& it = items[T.item];
    const int tree = it.tree;
    for (int64_t t = T.t0 + threadIdx.x; t < T.t1; t += blockDim.x) {
      switch (tree) {
        case 0: eval_sites<cat::MM, M, P_F64>(it.k, t, T.mu); break;
        case 1: eval_sites<cat::E1, M, P_F64>(it.k, t, T.mu); break;
        case 2: eval_sites<cat::MV, M, P_F64>(it.k, t, T.mu); break;
        case 3: eval_sites<cat::E2, M, P_F64>(it.k, t, T.mu); break;
        case 4: eval_sites<cat::E3, M, P_F64>(it.k, t, T.mu); break;
        case 5: eval_sites<cat::MMM, M, P_F64>(it.k, t, T.mu); break;
        case 6: eval_sites<cat::E1Lin, M, P_F64>(it.k, t, T.mu); break;
        default: eval_sites<cat::AdjMM, M, P_F64>(it.k, t, T.mu); break;
      }
    }
  }
}

}  // namespace su3s

using namespace su3s;

struct su3s_batch {
  struct Item {
    su3s_field* dest;
    const su3s_expr* e;
  };
  std::vector<Item> items;
  bool built = false;
  BItem* d_items = nullptr;
  BTile* d_tiles = nullptr;
  int64_t ntiles = 0, nsites = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static void batch_release(su3s_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_tiles) cudaFree(b->d_tiles);
  b->exec = nullptr;
  b->graph = nullptr;
  b->d_items = nullptr;
  b->d_tiles = nullptr;
}

SU3S_EXPORT int su3s_batch_create(su3s_batch** out) {
  if (!out) return fail(SU3S_EINVAL, "null output handle");
  *out = new (std::nothrow) su3s_batch;
  if (!*out) return fail(SU3S_ENOMEM, "out of host memory");
  return SU3S_OK;
}

SU3S_EXPORT int su3s_batch_add(su3s_batch* b, su3s_field* dest, const su3s_expr* e) {
  if (!b || !dest || !e) return fail(SU3S_EINVAL, "null argument");
  if (b->built) return fail(SU3S_EINVAL, "batch is already built");
  if (dest->prec != SU3S_F64) return fail(SU3S_EUNSUPPORTED, "batched items use FP64 storage");
  Canon c;
  int rc = canonicalize(e, &c);
  if (rc) return rc;
  if (c.kind != dest->kind) return fail(SU3S_ETYPE, "destination kind differs from the tree's");
  for (su3s_field* f : c.leaves) {
    rc = check_same_shape(f, dest, true);
    if (rc) return rc;
  }
  const_cast<su3s_expr*>(e)->ref.fetch_add(1);
  b->items.push_back({dest, e});
  return SU3S_OK;
}

SU3S_EXPORT int su3s_batch_build(su3s_batch* b, int math, int threads, int tile_sites,
                                 void* stream) {
  if (!b) return fail(SU3S_EINVAL, "null batch");
  if (b->built) return fail(SU3S_EINVAL, "batch is already built");
  if (threads == 0) threads = 256;
  if (threads < 32 || threads > 256 || threads % 32)
    return fail(SU3S_EINVAL, "threads per block must be a multiple of 32 in 32..256");
  if (tile_sites == 0) tile_sites = 4 * threads;
  if (tile_sites < threads) return fail(SU3S_EINVAL, "tile smaller than a block");
  if (!valid_math(math))
    return fail(SU3S_EINVAL, "bad arithmetic %d", math);
  int m = resolve_math(SU3S_F64, math);
  (void)stream;

  std::vector<BItem> hitems;
  std::vector<BTile> htiles;
  std::vector<size_t> others;  // item indices launched separately
  int64_t nsites = 0;
  for (size_t i = 0; i < b->items.size(); ++i) {
    Canon c;
    canonicalize(b->items[i].e, &c);
    int tree = -1;
    for (int t = 0; t < kNumBatchTrees; ++t)
      if (c.sig == kBatchTrees[t]) tree = t;
    nsites += b->items[i].dest->Vpad * b->items[i].dest->nmu;
    if (tree < 0) {
      others.push_back(i);
      continue;
    }
    BItem it;
    memset(&it, 0, sizeof it);
    build_params(c, b->items[i].dest, 1, &it.k);
    it.tree = tree;
    const int32_t idx = (int32_t)hitems.size();
    hitems.push_back(it);
    for (int mu = 0; mu < it.k.nmu; ++mu)
      for (int64_t t0 = 0; t0 < it.k.nvec; t0 += tile_sites) {
        int64_t t1 = t0 + tile_sites < it.k.nvec ? t0 + tile_sites : it.k.nvec;
        htiles.push_back(BTile{idx, mu, t0, t1});
      }
  }
  b->nsites = nsites;
  b->ntiles = (int64_t)htiles.size();

  cudaError_t ce;
  if (!hitems.empty()) {
    ce = cudaMalloc(&b->d_items, hitems.size() * sizeof(BItem));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_tiles, htiles.size() * sizeof(BTile));
    if (ce != cudaSuccess) {
      batch_release(b);
      return fail(SU3S_ENOMEM, "batch tables: %s", cudaGetErrorString(ce));
    }
    ce = cudaMemcpy(b->d_items, hitems.data(), hitems.size() * sizeof(BItem), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess)
      ce = cudaMemcpy(b->d_tiles, htiles.data(), htiles.size() * sizeof(BTile), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
      batch_release(b);
      return cuda_fail(ce, "batch table upload");
    }
  }

  // persistent grid from occupancy
  const void* kern = m == MATH_F64  ? (const void*)&k_batch<MathF64>
                     : m == MATH_FX ? (const void*)&k_batch<MathFX>
                                    : (const void*)&k_batch<MathDF>;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)per_sm * sm_count();
  if (grid > b->ntiles) grid = b->ntiles;
  if (grid < 1) grid = 1;

  cudaStream_t cap;
  ce = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (ce != cudaSuccess) {
    batch_release(b);
    return cuda_fail(ce, "capture stream");
  }
  ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  int rc = SU3S_OK;
  if (ce == cudaSuccess) {
    if (b->ntiles > 0) {
      if (m == MATH_F64) k_batch<MathF64><<<(unsigned)grid, threads, 0, cap>>>(b->d_items, b->d_tiles, b->ntiles);
      else if (m == MATH_FX) k_batch<MathFX><<<(unsigned)grid, threads, 0, cap>>>(b->d_items, b->d_tiles, b->ntiles);
      else k_batch<MathDF><<<(unsigned)grid, threads, 0, cap>>>(b->d_items, b->d_tiles, b->ntiles);
      ce = cudaGetLastError();
      if (ce != cudaSuccess) rc = cuda_fail(ce, "persistent kernel capture");
    }
    for (size_t i : others) {
      if (rc) break;
      rc = su3s_eval_math(b->items[i].dest, b->items[i].e, math, cap);
    }
    cudaGraph_t g = nullptr;
    cudaError_t ce2 = cudaStreamEndCapture(cap, &g);
    if (!rc && ce2 != cudaSuccess) rc = cuda_fail(ce2, "end of graph capture");
    if (!rc) {
      b->graph = g;
      ce2 = cudaGraphInstantiate(&b->exec, g, 0);
      if (ce2 != cudaSuccess) rc = cuda_fail(ce2, "graph instantiation");
    } else if (g) {
      cudaGraphDestroy(g);
    }
  } else {
    rc = cuda_fail(ce, "begin graph capture");
  }
  cudaStreamDestroy(cap);
  if (rc) {
    batch_release(b);
    return rc;
  }
  b->built = true;
  return SU3S_OK;
}

SU3S_EXPORT int su3s_batch_launch(su3s_batch* b, void* stream) {
  if (!b) return fail(SU3S_EINVAL, "null batch");
  if (!b->built) return fail(SU3S_EINVAL, "batch is not built");
  cudaError_t ce = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "graph launch");
  return SU3S_OK;
}

SU3S_EXPORT int su3s_batch_info(const su3s_batch* b, int64_t* sites, int64_t* tiles) {
  if (!b) return fail(SU3S_EINVAL, "null batch");
  if (sites) *sites = b->nsites;
  if (tiles) *tiles = b->ntiles;
  return SU3S_OK;
}

SU3S_EXPORT int su3s_batch_destroy(su3s_batch* b) {
  if (!b) return SU3S_OK;
  batch_release(b);
  for (auto& it : b->items) su3s_expr_free(const_cast<su3s_expr*>(it.e));
  delete b;
  return SU3S_OK;
}
