// Batched evaluation: many (destination, tree) items over lattices of uneven
// volumes run in persistent kernels, one per tree present in the batch (each
// compiled for its tree alone, so its register use is that tree's).  The host
// cuts every item into tiles of site vectors and groups the tiles by tree; for
// each group a fixed grid of blocks (sized from occupancy) walks its tile list
// round-robin.  These launches, plus separate launches for items whose tree no
// persistent kernel covers, are captured once into a CUDA graph and replayed
// with a single cudaGraphLaunch.
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

// At most 128 registers: two 256-thread blocks (16 warps) per SM.  The
// item's parameters are copied to shared memory once per tile, so the site
// loop reads them with broadcast shared-memory loads.
template <class M, class Tree>
__global__ void __launch_bounds__(256, 2) k_batch(const BItem* __restrict__ items,
                                                  const BTile* __restrict__ tiles, int64_t ntiles) {
  __shared__ KParams sk;
  constexpr int kWords = (int)(sizeof(KParams) / 4);
  static_assert(sizeof(KParams) % 4 == 0, "KParams is copied as 32-bit words");
  for (int64_t i = blockIdx.x; i < ntiles; i += gridDim.x) {
    const BTile T = tiles[i];
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&items[T.item].k);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sk);
    for (int w = threadIdx.x; w < kWords; w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    for (int64_t t = T.t0 + threadIdx.x; t < T.t1; t += blockDim.x)
      eval_sites<Tree, M, P_F64>(sk, t, T.mu);
    __syncthreads();
  }
}

// A 32-site tile of one item for the staged kernel.
struct BWTile {
  int32_t item;
  int32_t mu;
  int64_t s0;
};

// Staged persistent kernel: every warp takes a contiguous run of the list of
// 32-site tiles of all items (so consecutive tiles mostly share an item and
// its descriptors stay in L1) and walks it with the whole-tile TMA pipeline of
// the single-lattice kernels: one tensor copy per object, the next tile's
// copies in flight while the current one is computed.  Tensor maps and
// descriptors are read from the item table in global memory.
template <class M, class Tree>
__global__ void __launch_bounds__(256) k_batch_tma(const BItem* __restrict__ items,
                                                   const BWTile* __restrict__ wt, int64_t n,
                                                   int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (!smem_aligned(smem, err)) return;
  constexpr int NL = Tree::nleaf;
  constexpr int NS = Tree::nsc;
  constexpr int W = Width<Tree::kind>::value;
  constexpr int TB = TileBytes<Tree, P_F64, false>::value;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* buf = smem + warp * tma_warp_stride(TB);
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf + TB);
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t chunk = (n + nwarps - 1) / nwarps;
  int64_t i = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * chunk;
  const int64_t end = i + chunk < n ? i + chunk : n;
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncwarp();
  BWTile T{0, 0, 0};
  if (i < end) {
    T = wt[i];
    issue_tile<Tree, P_F64, false>(lane, items[T.item].k, nullptr, nullptr, T.s0, T.mu, buf, bar);
  }
  uint32_t phase = 0;
  Ctx<M, NL, NS> ctx;
  while (i < end) {
    const int64_t in = i + 1;
    const BWTile Tn = in < end ? wt[in] : T;   // read while this tile's copies land
    const KParams& p = items[T.item].k;
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, phase));
    if (!ok) {
      if (lane == 0) report_timeout(err, bar, phase);
      break;
    }
    phase ^= 1;
    ctx.gmax = p.gscal;
    if constexpr (TwoProducts<Tree>::value) {
      // the first product's leaves, the product, then the second's (as the
      // whole-tile single-lattice kernel)
      using TP = TwoProducts<Tree>;
      typename M::A acc[1][W];
      read_leaves_of<Tree, typename TP::P0, 0, P_F64, M>(buf, lane, ctx);
      acc_into<typename TP::P0, M, true, 1>(ctx, acc[0]);
      read_leaves_of<Tree, typename TP::P1, 0, P_F64, M>(buf, lane, ctx);
      fence_proxy_async_smem();
      __syncwarp();
      if (in < end)
        issue_tile<Tree, P_F64, false>(lane, items[Tn.item].k, nullptr, nullptr, Tn.s0, Tn.mu, buf, bar);
      if (M::kGuard && __any_sync(0xffffffffu, guard_trips<Tree>(ctx.gmax))) {
        eval_site_f64<Tree, P_F64>(p, T.s0 + lane, T.mu);
      } else {
        mul_combine<M, TP::S1>(ctx, acc[0], (typename TP::P1*)nullptr);
        store_obj<Tree::kind, P_F64, M, 1, W>(p.dst, T.s0 + lane, T.mu, acc);
      }
      T = Tn;
      i = in;
      continue;
    }
    read_leaves<Tree, 0, P_F64, M>(buf, lane, ctx);
    fence_proxy_async_smem();
    __syncwarp();
    if (in < end)
      issue_tile<Tree, P_F64, false>(lane, items[Tn.item].k, nullptr, nullptr, Tn.s0, Tn.mu, buf, bar);
#pragma unroll
    for (int k = 0; k < (NS > 0 ? NS : 1); ++k) ctx.sc[k] = M::scalar(p.sc[k], p.sch[k], p.scl[k]);
    if (M::kGuard && __any_sync(0xffffffffu, guard_trips<Tree>(ctx.gmax))) {
      eval_site_f64<Tree, P_F64>(p, T.s0 + lane, T.mu);
    } else {
      typename M::A acc[1][W];
      acc_into<Tree, M, true, 1>(ctx, acc[0]);
      store_obj<Tree::kind, P_F64, M, 1, W>(p.dst, T.s0 + lane, T.mu, acc);
    }
    T = Tn;
    i = in;
  }
}

// Persistent kernel of batch tree `tree` in arithmetic M.
template <class M>
static const void* batch_kernel(int tree) {
  switch (tree) {
    case 0: return (const void*)&k_batch<M, cat::MM>;
    case 1: return (const void*)&k_batch<M, cat::E1>;
    case 2: return (const void*)&k_batch<M, cat::MV>;
    case 3: return (const void*)&k_batch<M, cat::E2>;
    case 4: return (const void*)&k_batch<M, cat::E3>;
    case 5: return (const void*)&k_batch<M, cat::MMM>;
    case 6: return (const void*)&k_batch<M, cat::E1Lin>;
    default: return (const void*)&k_batch<M, cat::AdjMM>;
  }
}

static const void* batch_kernel(int math, int tree) {
  return math == MATH_F64  ? batch_kernel<MathF64>(tree)
         : math == MATH_FX ? batch_kernel<MathFX>(tree)
                           : batch_kernel<MathDF>(tree);
}

// Staged persistent kernel of batch tree `tree` and its tile bytes per warp.
template <class M, class Tree>
static const void* staged_entry(int* warp_bytes) {
  *warp_bytes = tma_warp_stride(TileBytes<Tree, P_F64, false>::value);
  return (const void*)&k_batch_tma<M, Tree>;
}
template <class M>
static const void* batch_kernel_tma(int tree, int* warp_bytes) {
  switch (tree) {
    case 0: return staged_entry<M, cat::MM>(warp_bytes);
    case 1: return staged_entry<M, cat::E1>(warp_bytes);
    case 2: return staged_entry<M, cat::MV>(warp_bytes);
    case 3: return staged_entry<M, cat::E2>(warp_bytes);
    case 4: return staged_entry<M, cat::E3>(warp_bytes);
    case 5: return staged_entry<M, cat::MMM>(warp_bytes);
    case 6: return staged_entry<M, cat::E1Lin>(warp_bytes);
    default: return staged_entry<M, cat::AdjMM>(warp_bytes);
  }
}
static const void* batch_kernel_tma(int math, int tree, int* warp_bytes) {
  return math == MATH_F64  ? batch_kernel_tma<MathF64>(tree, warp_bytes)
         : math == MATH_FX ? batch_kernel_tma<MathFX>(tree, warp_bytes)
                           : batch_kernel_tma<MathDF>(tree, warp_bytes);
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
  BWTile* d_wtiles = nullptr;   // 32-site tiles of the staged items
  int64_t ntiles = 0, nsites = 0;
  int64_t nplain = 0;   // tiles of the plain-load kernels (the tile size matters only for these)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static bool overlaps(const su3s_field* a, const su3s_field* b) {
  const char* pa = (const char*)a->ptr;
  const char* pb = (const char*)b->ptr;
  return pa < pb + b->bytes && pb < pa + a->bytes;
}

static void batch_release(su3s_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_wtiles) cudaFree(b->d_wtiles);
  b->exec = nullptr;
  b->graph = nullptr;
  b->d_items = nullptr;
  b->d_tiles = nullptr;
  b->d_wtiles = nullptr;
  b->built = false;
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

// Items run concurrently: no item may write memory another item reads or writes.
static int check_independent(const su3s_batch* b) {
  for (size_t i = 0; i < b->items.size(); ++i) {
    const su3s_field* di = b->items[i].dest;
    for (size_t j = 0; j < b->items.size(); ++j) {
      if (j == i) continue;
      Canon cj;
      if (canonicalize(b->items[j].e, &cj)) continue;
      const su3s_field* dj = b->items[j].dest;
      bool clash = overlaps(di, dj);
      for (const su3s_field* f : cj.leaves) clash = clash || overlaps(di, f);
      if (clash)
        return fail(SU3S_EINVAL, "batch item %zu writes memory that item %zu reads or writes", i, j);
    }
  }
  return SU3S_OK;
}

// Tables, grids and graph of batch b (arguments checked by the caller);
// blocks_per_sm caps the persistent grids (0: as many as fit).
static int batch_build(su3s_batch* b, int math, int threads, int tile_sites, int blocks_per_sm) {
  const int m = resolve_math(SU3S_F64, math);
  std::vector<BItem> hitems;
  std::vector<BTile> by_tree[kNumBatchTrees];     // plain-load tiles
  std::vector<BWTile> staged_by_tree[kNumBatchTrees];  // 32-site tiles of staged items
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
    const bool staged = tma_tree_ok(c, b->items[i].dest) && it.k.nvec % 32 == 0;
    for (int mu = 0; mu < it.k.nmu; ++mu) {
      if (staged) {
        for (int64_t s0 = 0; s0 < it.k.nvec; s0 += 32)
          staged_by_tree[tree].push_back(BWTile{idx, mu, s0});
        continue;
      }
      for (int64_t t0 = 0; t0 < it.k.nvec; t0 += tile_sites) {
        int64_t t1 = t0 + tile_sites < it.k.nvec ? t0 + tile_sites : it.k.nvec;
        by_tree[tree].push_back(BTile{idx, mu, t0, t1});
      }
    }
  }
  // tiles grouped by tree: group t is htiles[first[t], first[t] + count[t])
  std::vector<BTile> htiles;
  int64_t first[kNumBatchTrees], count[kNumBatchTrees];
  for (int t = 0; t < kNumBatchTrees; ++t) {
    first[t] = (int64_t)htiles.size();
    count[t] = (int64_t)by_tree[t].size();
    htiles.insert(htiles.end(), by_tree[t].begin(), by_tree[t].end());
  }
  std::vector<BWTile> hwtiles;
  int64_t wfirst[kNumBatchTrees], wcount[kNumBatchTrees];
  for (int t = 0; t < kNumBatchTrees; ++t) {
    wfirst[t] = (int64_t)hwtiles.size();
    wcount[t] = (int64_t)staged_by_tree[t].size();
    hwtiles.insert(hwtiles.end(), staged_by_tree[t].begin(), staged_by_tree[t].end());
  }
  b->nsites = nsites;
  b->ntiles = (int64_t)htiles.size() + (int64_t)hwtiles.size();
  b->nplain = (int64_t)htiles.size();

  cudaError_t ce;
  if (!hitems.empty()) {
    ce = cudaMalloc(&b->d_items, hitems.size() * sizeof(BItem));
    if (ce == cudaSuccess && !htiles.empty())
      ce = cudaMalloc(&b->d_tiles, htiles.size() * sizeof(BTile));
    if (ce == cudaSuccess && !hwtiles.empty())
      ce = cudaMalloc(&b->d_wtiles, hwtiles.size() * sizeof(BWTile));
    if (ce != cudaSuccess) {
      batch_release(b);
      return fail(SU3S_ENOMEM, "batch tables: %s", cudaGetErrorString(ce));
    }
    ce = cudaMemcpy(b->d_items, hitems.data(), hitems.size() * sizeof(BItem), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && !htiles.empty())
      ce = cudaMemcpy(b->d_tiles, htiles.data(), htiles.size() * sizeof(BTile), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && !hwtiles.empty())
      ce = cudaMemcpy(b->d_wtiles, hwtiles.data(), hwtiles.size() * sizeof(BWTile),
                      cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
      batch_release(b);
      return cuda_fail(ce, "batch table upload");
    }
  }

  // staged groups: persistent grid from occupancy with the warps' tile buffers
  int64_t wgrid[kNumBatchTrees];
  size_t wsmem[kNumBatchTrees];
  for (int t = 0; t < kNumBatchTrees; ++t) {
    wgrid[t] = 1;
    wsmem[t] = 0;
    if (wcount[t] == 0) continue;
    int wb = 0;
    const void* k = batch_kernel_tma(m, t, &wb);
    wsmem[t] = (size_t)(threads / 32) * wb;
    int per_sm = 1;
    ce = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem[t]);
    if (ce == cudaSuccess)
      ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, wsmem[t]);
    if (ce != cudaSuccess) {
      batch_release(b);
      return cuda_fail(ce, "staged batch kernel setup");
    }
    if (blocks_per_sm > 0 && per_sm > blocks_per_sm) per_sm = blocks_per_sm;
    if (per_sm < 1) per_sm = 1;
    const int64_t warps = (int64_t)per_sm * sm_count() * (threads / 32);
    int64_t blocks = (int64_t)per_sm * sm_count();
    if (warps > wcount[t]) blocks = (wcount[t] + threads / 32 - 1) / (threads / 32);
    wgrid[t] = blocks < 1 ? 1 : blocks;
  }

  // persistent grid of each group from its kernel's occupancy
  int64_t grid[kNumBatchTrees];
  for (int t = 0; t < kNumBatchTrees; ++t) {
    int per_sm = 1;
    if (count[t] > 0)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel(m, t), threads, 0);
    if (blocks_per_sm > 0 && per_sm > blocks_per_sm) per_sm = blocks_per_sm;
    if (per_sm < 1) per_sm = 1;
    grid[t] = (int64_t)per_sm * sm_count();
    if (grid[t] > count[t]) grid[t] = count[t];
    if (grid[t] < 1) grid[t] = 1;
  }

  cudaStream_t cap;
  ce = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (ce != cudaSuccess) {
    batch_release(b);
    return cuda_fail(ce, "capture stream");
  }
  ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  int rc = SU3S_OK;
  if (ce == cudaSuccess) {
    int* err = hitems.empty() ? nullptr : hitems[0].k.err;   // the library's device error word
    for (int t = 0; t < kNumBatchTrees && !rc; ++t) {
      if (wcount[t] == 0) continue;
      int wb = 0;
      const BItem* items = b->d_items;
      const BWTile* wt = b->d_wtiles + wfirst[t];
      int64_t n = wcount[t];
      void* args[] = {(void*)&items, (void*)&wt, (void*)&n, (void*)&err};
      ce = cudaLaunchKernel(batch_kernel_tma(m, t, &wb), dim3((unsigned)wgrid[t]),
                            dim3((unsigned)threads), args, wsmem[t], cap);
      if (ce != cudaSuccess) rc = cuda_fail(ce, "staged persistent kernel capture");
    }
    for (int t = 0; t < kNumBatchTrees && !rc; ++t) {
      if (count[t] == 0) continue;
      const BItem* items = b->d_items;
      const BTile* tiles = b->d_tiles + first[t];
      int64_t n = count[t];
      void* args[] = {(void*)&items, (void*)&tiles, (void*)&n};
      ce = cudaLaunchKernel(batch_kernel(m, t), dim3((unsigned)grid[t]), dim3((unsigned)threads),
                            args, 0, cap);
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

static int check_build_args(int math, int threads, int tile_sites) {
  if (threads < 32 || threads > 256 || threads % 32)
    return fail(SU3S_EINVAL, "threads per block must be a multiple of 32 in 32..256");
  if (tile_sites < threads) return fail(SU3S_EINVAL, "tile smaller than a block");
  if (!valid_math(math)) return fail(SU3S_EINVAL, "bad arithmetic %d", math);
  return SU3S_OK;
}

SU3S_EXPORT int su3s_batch_build(su3s_batch* b, int math, int threads, int tile_sites,
                                 void* stream) {
  if (!b) return fail(SU3S_EINVAL, "null batch");
  if (b->built) return fail(SU3S_EINVAL, "batch is already built");
  if (threads == 0) threads = 256;
  if (tile_sites == 0) tile_sites = 2 * threads;
  int rc = check_build_args(math, threads, tile_sites);
  if (!rc) rc = check_independent(b);
  if (rc) return rc;
  (void)stream;
  return batch_build(b, math, threads, tile_sites, 0);
}

SU3S_EXPORT int su3s_batch_tune(su3s_batch* b, int math, void* stream, int* threads_out,
                                int* tile_sites_out, int* bps_out, float* best_ms) {
  if (!b) return fail(SU3S_EINVAL, "null batch");
  int rc = check_build_args(math, 256, 512);
  if (!rc) rc = check_independent(b);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fail(SU3S_ECUDA, "event creation failed");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(SU3S_ECUDA, "event creation failed");
  }
  const int th_c[] = {64, 128, 256};
  const int bps_c[] = {0, 1, 2, 4};
  const int tile_c[] = {2, 1, 4};   // tile = multiple of the block (plain-load tiles only)
  float best = 1e30f;
  int bt = 256, btile = 512, bb = 0;
  bool plain = true;   // known after the first build
  for (int th : th_c) {
    for (int bps : bps_c) {
      for (int tm : tile_c) {
        if (!plain && tm != 2) continue;
        batch_release(b);
        rc = batch_build(b, math, th, tm * th, bps);
        if (rc) break;
        plain = b->nplain > 0;
        cudaError_t ce = cudaGraphLaunch(b->exec, st);   // warm-up
        float ms = 1e30f;
        for (int trial = 0; trial < 2 && ce == cudaSuccess; ++trial) {
          ce = cudaEventRecord(e0, st);
          for (int r = 0; r < 3 && ce == cudaSuccess; ++r) ce = cudaGraphLaunch(b->exec, st);
          if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
          if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
          float t = 0.f;
          if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
          if (ce == cudaSuccess && t / 3.f < ms) ms = t / 3.f;
        }
        if (ce != cudaSuccess) {
          rc = cuda_fail(ce, "batch tuning launch");
          break;
        }
        if (ms < best) {
          best = ms;
          bt = th;
          btile = tm * th;
          bb = bps;
        }
      }
      if (rc) break;
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  batch_release(b);
  if (rc) return rc;
  rc = batch_build(b, math, bt, btile, bb);
  if (rc) return rc;
  if (threads_out) *threads_out = bt;
  if (tile_sites_out) *tile_sites_out = btile;
  if (bps_out) *bps_out = bb;
  if (best_ms) *best_ms = best;
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
