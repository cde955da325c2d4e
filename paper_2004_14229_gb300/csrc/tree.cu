// Uniform box cluster trees on the device (Alg. 1, Sect. 2.1).
//
// Alg. 1 bisects a box at its centre c and sends a point to the lower child
// when x <= c, to the upper one when x > c.  Every point's descent is
// therefore fixed by its depth-D cell, which we compute by the same bisection
// in FP64 (bit-identical to the recursion), encode as a Morton key (x in bit
// 0, child index bx + 2 by + 4 bz), and sort stably with the original index
// as payload.  Boxes of level l are the runs of equal key >> 3 (D - l); a run
// keeps its points in ascending original index because the sort is stable.
#include <algorithm>
#include <cstring>

#include "dfdm_internal.cuh"

namespace dfdm {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// ------------------------------------------------------------------ scan
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of one 4096-element tile; writes the tile total to bsum.
__global__ void k_scan_tile(const uint32_t *in, uint32_t *out, int64_t n,
                            uint32_t *bsum) {
  __shared__ uint32_t wsum[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t t = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0u;
    t += v[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = warp_incl_scan(t);
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = wsum[lane];
    wsum[lane] = warp_incl_scan(s) - s;  // exclusive warp offsets
  }
  __syncthreads();
  uint32_t run = incl - t + wsum[warp];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = run;
}

__global__ void k_scan_add(uint32_t *out, int64_t n, const uint32_t *boff) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += boff[i / kScanTile];
}

// Exclusive prefix sum in place-or-not; returns the total.
uint32_t exclusive_scan(Plan &plan, const uint32_t *in, uint32_t *out, int64_t n,
                        cudaStream_t st) {
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  uint32_t *bsum = nullptr, *boff = nullptr;
  DFDM_CUDA_TRY(cudaMalloc(&bsum, (nb + 1) * sizeof(uint32_t)));
  DFDM_CUDA_TRY(cudaMalloc(&boff, (nb + 1) * sizeof(uint32_t)));
  k_scan_tile<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, bsum);
  DFDM_LAUNCH_CHECK();
  uint32_t total = 0;
  if (nb > 1) {
    total = exclusive_scan(plan, bsum, boff, nb, st);
    k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, boff);
    DFDM_LAUNCH_CHECK();
  } else {
    DFDM_CUDA_TRY(cudaMemcpyAsync(&total, bsum, sizeof(uint32_t),
                                  cudaMemcpyDeviceToHost, st));
    DFDM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  cudaFree(bsum);
  cudaFree(boff);
  return total;
}

// ------------------------------------------------------------- Morton keys
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | x << 32) & 0x1f00000000ffffull;
  x = (x | x << 16) & 0x1f0000ff0000ffull;
  x = (x | x << 8) & 0x100f00f00f00f00full;
  x = (x | x << 4) & 0x10c30c30c30c30c3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x1fffffull;
  return (uint32_t)x;
}

// Cell of every point on the depth-D grid by Alg. 1's bisection, as a key.
__global__ void k_morton(const double *pts, int64_t n, double lo0, double lo1,
                         double lo2, double side, int depth, uint64_t *keys,
                         int32_t *idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double lo_root[3] = {lo0, lo1, lo2};
  uint32_t cell[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double x = pts[3 * i + a];
    double lo = lo_root[a], hi = lo_root[a] + side;
    uint32_t c = 0;
    for (int l = 0; l < depth; ++l) {
      const double mid = (lo + hi) / 2.0;   // centre of Alg. 1
      if (x > mid) {                        // (mid, hi] -> upper child
        c = (c << 1) | 1u;
        lo = mid;
      } else {                              // (lo, mid] -> lower child
        c = c << 1;
        hi = mid;
      }
    }
    cell[a] = c;
  }
  keys[i] = spread3(cell[0]) | (spread3(cell[1]) << 1) | (spread3(cell[2]) << 2);
  idx[i] = (int32_t)i;
}

// ------------------------------------------------------------ radix sort
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 16;
constexpr int kRsTile = kRsThreads * kRsRounds;   // 4096 keys per tile

__global__ void k_rs_hist(const uint64_t *keys, int64_t n, int shift,
                          uint32_t *hist, int ntiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
    if (base + i < n) atomicAdd(&h[(keys[base + i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: warp w ranks its 512 keys in 16 ordered rounds.
__global__ void k_rs_scatter(const uint64_t *kin, const int32_t *vin,
                             uint64_t *kout, int32_t *vout, int64_t n, int shift,
                             const uint32_t *offs, int ntiles) {
  __shared__ uint32_t wcnt[kRsWarps][257];
  __shared__ uint32_t woff[kRsWarps][257];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRsWarps * 257; i += kRsThreads) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile + warp * (kRsTile / kRsWarps);
  uint32_t local[kRsRounds];
  uint32_t digit[kRsRounds];
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    const int64_t i = base + r * 32 + lane;
    const bool valid = i < n;
    const uint32_t d = valid ? (uint32_t)((kin[i] >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = wcnt[warp][d];
    __syncwarp();
    if (lane == __ffs(peers) - 1) wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
    local[r] = before + __popc(peers & lt_mask);
    digit[r] = d;
  }
  __syncthreads();
  {
    const int d = threadIdx.x;  // 256 threads, one digit each
    uint32_t run = 0;
    for (int w = 0; w < kRsWarps; ++w) {
      woff[w][d] = run;
      run += wcnt[w][d];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    const int64_t i = base + r * 32 + lane;
    if (i < n) {
      const uint32_t d = digit[r];
      const uint32_t pos = offs[(int64_t)d * ntiles + blockIdx.x] + woff[warp][d] + local[r];
      kout[pos] = kin[i];
      vout[pos] = vin[i];
    }
  }
}

void radix_sort(Plan &plan, uint64_t *&keys, int32_t *&vals, int64_t n, int bits,
                cudaStream_t st) {
  const int ntiles = (int)((n + kRsTile - 1) / kRsTile);
  uint64_t *k2 = nullptr;
  int32_t *v2 = nullptr;
  uint32_t *hist = nullptr, *offs = nullptr;
  DFDM_CUDA_TRY(cudaMalloc(&k2, n * sizeof(uint64_t)));
  DFDM_CUDA_TRY(cudaMalloc(&v2, n * sizeof(int32_t)));
  DFDM_CUDA_TRY(cudaMalloc(&hist, (size_t)256 * ntiles * sizeof(uint32_t)));
  DFDM_CUDA_TRY(cudaMalloc(&offs, (size_t)256 * ntiles * sizeof(uint32_t)));
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<<<ntiles, kRsThreads, 0, st>>>(keys, n, shift, hist, ntiles);
    DFDM_LAUNCH_CHECK();
    exclusive_scan(plan, hist, offs, (int64_t)256 * ntiles, st);
    k_rs_scatter<<<ntiles, kRsThreads, 0, st>>>(keys, vals, k2, v2, n, shift, offs, ntiles);
    DFDM_LAUNCH_CHECK();
    std::swap(keys, k2);
    std::swap(vals, v2);
  }
  DFDM_CUDA_TRY(cudaStreamSynchronize(st));
  cudaFree(k2);
  cudaFree(v2);
  cudaFree(hist);
  cudaFree(offs);
}

// --------------------------------------------------------- level boxes
__global__ void k_run_flags(const uint64_t *keys, int64_t n, int shift,
                            uint32_t *flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  flag[i] = (i == 0 || (keys[i] >> shift) != (keys[i - 1] >> shift)) ? 1u : 0u;
}

__global__ void k_run_starts(const uint64_t *keys, int64_t n, int shift,
                             const uint32_t *flag, const uint32_t *pos,
                             int32_t *begin, uint64_t *boxkey) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !flag[i]) return;
  begin[pos[i]] = (int32_t)i;
  boxkey[pos[i]] = keys[i] >> shift;
}

__global__ void k_run_ends(const int32_t *begin, int64_t nb, int64_t n,
                           int32_t *end) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  end[b] = (b + 1 < nb) ? begin[b + 1] : (int32_t)n;
}

__global__ void k_gather_xyz(const double *pts, const int32_t *perm, int64_t n,
                             double *xyz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t j = perm[i];
  xyz[i] = pts[3 * (int64_t)j];
  xyz[n + i] = pts[3 * (int64_t)j + 1];
  xyz[2 * n + i] = pts[3 * (int64_t)j + 2];
}

__global__ void k_leaf_cells(const uint64_t *boxkey, int64_t nb, int level,
                             int32_t *cell, int32_t *leaf_of_cell) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const uint64_t k = boxkey[b];
  const uint32_t x = compact3(k), y = compact3(k >> 1), z = compact3(k >> 2);
  const int64_t g = 1ll << level;
  const int64_t c = x + g * (y + g * (int64_t)z);
  cell[b] = (int32_t)c;
  leaf_of_cell[c] = (int32_t)b;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Boxes of one level: begin/end in sorted order and their keys (device).
int64_t level_boxes(Plan &plan, const Tree &tree, int level, int32_t *&begin,
                    int32_t *&end, uint64_t *&boxkey, cudaStream_t st) {
  const int64_t n = tree.n;
  const int shift = 3 * (tree.key_depth - level);
  uint32_t *flag = nullptr, *pos = nullptr;
  DFDM_CUDA_TRY(cudaMalloc(&flag, n * sizeof(uint32_t)));
  DFDM_CUDA_TRY(cudaMalloc(&pos, n * sizeof(uint32_t)));
  k_run_flags<<<blocks_for(n, 256), 256, 0, st>>>(tree.keys, n, shift, flag);
  DFDM_LAUNCH_CHECK();
  const int64_t nb = exclusive_scan(plan, flag, pos, n, st);
  DFDM_CUDA_TRY(cudaMalloc(&begin, nb * sizeof(int32_t)));
  DFDM_CUDA_TRY(cudaMalloc(&end, nb * sizeof(int32_t)));
  DFDM_CUDA_TRY(cudaMalloc(&boxkey, nb * sizeof(uint64_t)));
  k_run_starts<<<blocks_for(n, 256), 256, 0, st>>>(tree.keys, n, shift, flag, pos, begin, boxkey);
  DFDM_LAUNCH_CHECK();
  k_run_ends<<<blocks_for(nb, 256), 256, 0, st>>>(begin, nb, n, end);
  DFDM_LAUNCH_CHECK();
  DFDM_CUDA_TRY(cudaStreamSynchronize(st));
  cudaFree(flag);
  cudaFree(pos);
  return nb;
}

}  // namespace

void build_tree(Plan &plan, Tree &tree, const double *host_pts, int64_t n,
                cudaStream_t st) {
  const int D = plan.params.max_depth;
  tree.n = n;
  tree.key_depth = D;
  double *pts = nullptr;
  DFDM_CUDA_TRY(cudaMalloc(&pts, n * 3 * sizeof(double)));
  DFDM_CUDA_TRY(cudaMemcpyAsync(pts, host_pts, n * 3 * sizeof(double),
                                cudaMemcpyHostToDevice, st));
  uint64_t *keys = nullptr;
  int32_t *idx = nullptr;
  DFDM_CUDA_TRY(cudaMalloc(&keys, n * sizeof(uint64_t)));
  DFDM_CUDA_TRY(cudaMalloc(&idx, n * sizeof(int32_t)));
  k_morton<<<blocks_for(n, 256), 256, 0, st>>>(pts, n, plan.root_lo[0], plan.root_lo[1],
                                               plan.root_lo[2], plan.root_side, D, keys, idx);
  DFDM_LAUNCH_CHECK();
  if (D > 0) radix_sort(plan, keys, idx, n, 3 * D, st);
  tree.keys = plan.alloc<uint64_t>(n);
  tree.perm = plan.alloc<int32_t>(n);
  DFDM_CUDA_TRY(cudaMemcpyAsync(tree.keys, keys, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
  DFDM_CUDA_TRY(cudaMemcpyAsync(tree.perm, idx, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  tree.xyz = plan.alloc<double>(3 * n);
  k_gather_xyz<<<blocks_for(n, 256), 256, 0, st>>>(pts, tree.perm, n, tree.xyz);
  DFDM_LAUNCH_CHECK();
  DFDM_CUDA_TRY(cudaStreamSynchronize(st));
  cudaFree(pts);
  cudaFree(keys);
  cudaFree(idx);

  // Depth p of Alg. 1: with n_max = 0 every non-empty box is refined to D.
  // Otherwise p is the first level whose boxes all hold <= n_max points; the
  // tree is uniform (all leaves on level p) iff no box above p is that small.
  int p = D;
  if (plan.params.n_max > 0) {
    p = -1;
    for (int l = 0; l <= D && p < 0; ++l) {
      int32_t *b = nullptr, *e = nullptr;
      uint64_t *k = nullptr;
      const int64_t nb = level_boxes(plan, tree, l, b, e, k, st);
      std::vector<int32_t> hb(nb), he(nb);
      DFDM_CUDA_TRY(cudaMemcpy(hb.data(), b, nb * sizeof(int32_t), cudaMemcpyDeviceToHost));
      DFDM_CUDA_TRY(cudaMemcpy(he.data(), e, nb * sizeof(int32_t), cudaMemcpyDeviceToHost));
      cudaFree(b);
      cudaFree(e);
      cudaFree(k);
      int32_t mx = 0, mn = INT32_MAX;
      for (int64_t i = 0; i < nb; ++i) {
        mx = std::max(mx, he[i] - hb[i]);
        mn = std::min(mn, he[i] - hb[i]);
      }
      if (mx <= plan.params.n_max || l == D) {
        p = l;
      } else if (mn <= plan.params.n_max) {
        throw Error{DFDM_ERR_UNSUPPORTED,
                    "the cluster tree of Alg. 1 is not of uniform depth (level " +
                        std::to_string(l) + " has leaves and non-leaves)"};
      }
    }
  }
  tree.depth = p;

  // Leaves on level p and the dense cell -> leaf lookup.
  int32_t *b = nullptr, *e = nullptr;
  uint64_t *k = nullptr;
  const int64_t nb = level_boxes(plan, tree, p, b, e, k, st);
  tree.nleaves = nb;
  tree.leaf_begin = plan.alloc<int32_t>(nb);
  tree.leaf_end = plan.alloc<int32_t>(nb);
  tree.leaf_cell = plan.alloc<int32_t>(nb);
  const int64_t ncell = 1ll << (3 * p);
  tree.leaf_of_cell = plan.alloc<int32_t>(ncell);
  DFDM_CUDA_TRY(cudaMemsetAsync(tree.leaf_of_cell, 0xff, ncell * sizeof(int32_t), st));
  DFDM_CUDA_TRY(cudaMemcpyAsync(tree.leaf_begin, b, nb * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  DFDM_CUDA_TRY(cudaMemcpyAsync(tree.leaf_end, e, nb * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  k_leaf_cells<<<blocks_for(nb, 256), 256, 0, st>>>(k, nb, p, tree.leaf_cell, tree.leaf_of_cell);
  DFDM_LAUNCH_CHECK();
  std::vector<int32_t> hb(nb), he(nb);
  DFDM_CUDA_TRY(cudaMemcpyAsync(hb.data(), b, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  DFDM_CUDA_TRY(cudaMemcpyAsync(he.data(), e, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  DFDM_CUDA_TRY(cudaStreamSynchronize(st));
  int32_t mx = 0;
  for (int64_t i = 0; i < nb; ++i) mx = std::max(mx, he[i] - hb[i]);
  tree.max_leaf_size = mx;
  cudaFree(b);
  cudaFree(e);
  cudaFree(k);
}

void export_level(const Plan &plan, const Tree &tree, int level,
                  std::vector<int64_t> &keys, std::vector<int64_t> &begin,
                  std::vector<int64_t> &end, cudaStream_t st) {
  int32_t *b = nullptr, *e = nullptr;
  uint64_t *k = nullptr;
  const int64_t nb = level_boxes(const_cast<Plan &>(plan), tree, level, b, e, k, st);
  std::vector<int32_t> hb(nb), he(nb);
  std::vector<uint64_t> hk(nb);
  DFDM_CUDA_TRY(cudaMemcpy(hb.data(), b, nb * sizeof(int32_t), cudaMemcpyDeviceToHost));
  DFDM_CUDA_TRY(cudaMemcpy(he.data(), e, nb * sizeof(int32_t), cudaMemcpyDeviceToHost));
  DFDM_CUDA_TRY(cudaMemcpy(hk.data(), k, nb * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  cudaFree(b);
  cudaFree(e);
  cudaFree(k);
  keys.assign(hk.begin(), hk.end());
  begin.assign(hb.begin(), hb.end());
  end.assign(he.begin(), he.end());
}

}  // namespace dfdm
