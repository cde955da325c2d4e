// Tensor-core form of Alg. 4 (DFDM_TC_FP16X3).
//
// M2L, the dense complex contraction g~_t += A~_d v~_{t-d} over all
// admissible offsets d (Sect. 2.6, multiplication phase; one stored operator
// per level and offset, Sect. 2.7), runs on the tcgen05 tensor cores
// (k_m2l_pair):
//   * complex n x n products are real-stacked: outputs [Re; Im] (N) times
//     inputs [Re v; Im v] (K), each padded to NP = KP (a multiple of 64);
//   * each value a is split into two FP16 terms a = a_hi + a_lo (a_hi =
//     fp16(a), a_lo = fp16(a - a_hi)) after a power-of-two scale per level,
//     and the product takes a_hi b_hi + a_lo b_hi + a_hi b_lo with FP32
//     accumulation in TMEM (the dropped a_lo b_lo is ~2^-22 relative);
//     H = M_hi O_hi lives for one unit of kPU stages (the accumulator is
//     truncated toward zero after every instruction), X = M_lo O_hi +
//     M_hi O_lo for kPXUnits units;
//   * a cluster of two CTAs owns 256 targets of one parity alpha (an
//     8 x 4 x 8 block of the parent grid) and walks one chunk of the level's
//     offset list for alpha with tcgen05.mma.cta_group::2 (M = 256, every row
//     a target; N = 224, one half of the stacked outputs per pass; each CTA
//     holds half of every operator tile);
//   * moments are split into a parity layout [slot][K step][parity][z/2]
//     [y/2][x/2][32], so a CTA's 128 source rows for offset d are one 5-D TMA
//     box (out-of-grid sources arrive as zeros); a CTA's share of an operator
//     stage is one 2-D TMA box of its pre-swizzled image; both CTAs' copies
//     complete on rank 0's per-unit "go" barrier (.cta_group::2);
//   * warp roles: 0 copies (both CTAs), 1 issues the MMAs (rank 0) and owns
//     TMEM (both), 2-13 drain H and X into FP32 running sums held in
//     registers and add them to the FP64 locals by coalesced atomics, one
//     32 x 16 slice every second unit.  Every wait is bounded; a wait that
//     gives up sets the plan's error word (read by dfdm_plan_check) and both
//     CTAs leave their loops.
//
// S2M and L2T run in FP64 (coordinates, Lagrange basis, plane waves, sums);
// M2M and L2L in FP32 with FP64 phase tables; the nearfield in FP32 on
// packed pairs (two sources per instruction) with FP64 totals.  Moments are
// real-stacked FP32 rows [Re 0..n-1 | Im 0..n-1 | pad] of KP floats, locals
// FP64 rows [Re 0..n-1 | pad | Im 0..n-1 | pad] with the imaginary part at
// KP / 2 (both halves start on 128-byte boundaries for the coalesced
// slice additions).
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "sm100_ptx.cuh"
#include "tc.cuh"

namespace dfdm {

namespace {

// This translation unit's copies of the reference nodes (FP64 and FP32) and
// barycentric factors; filled by build_tc.
__constant__ double c_cheb[kMaxOrder];
__constant__ double c_lagw[kMaxOrder];

constexpr double kPi = 3.14159265358979323846;


inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// ------------------------------------------------------------ helpers
// The o 1-D Lagrange basis values at t in [-1, 1] (reference nodes of Eq. 4,
// barycentric factors c_lagw), FP64.
template <int O>
__device__ __forceinline__ void lagrange1d(double t, double *out) {
#pragma unroll
  for (int nu = 0; nu < O; ++nu) {
    double v = c_lagw[nu];
#pragma unroll
    for (int mu = 0; mu < O; ++mu)
      if (mu != nu) v *= (t - c_cheb[mu]);
    out[nu] = v;
  }
}

// |v| with every non-finite value mapped to +inf (fmaxf would drop a NaN),
// so a level maximum shows that the level holds a non-finite moment
__device__ __forceinline__ float abs_or_inf(float v) {
  const float a = fabsf(v);
  return (a <= 3.402823466e38f) ? a : __int_as_float(0x7f800000);
}

__device__ __forceinline__ void atomic_max_abs(float *addr, float v) {
  atomicMax(reinterpret_cast<int *>(addr), __float_as_int(fabsf(v)));
}

// Centred directional diagonals P_{oct,c}[k] (FP64 arguments) as float2.
__global__ void k_phase_table_f(int order, int n, int nslots, const double *cvec, const double *c2vec,
                                double kappa, double h, float2 *tab) {
  const int oct = blockIdx.y, slot = blockIdx.x;
  const double b[3] = {(double)(oct & 1), (double)((oct >> 1) & 1), (double)((oct >> 2) & 1)};
  const double *c = cvec + 3 * slot, *c2 = c2vec + 3 * slot;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int kk[3] = {k % order, (k / order) % order, k / (order * order)};
    double a = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double r = c_cheb[kk[i]];
      a += (2.0 * b[i] - 1.0 + r) * c[i] - r * c2[i];
    }
    double s, co;
    sincos(kappa * h * a, &s, &co);
    tab[((int64_t)oct * nslots + slot) * n + k] = make_float2((float)co, (float)s);
  }
}

// Leaf-local FP32 coordinates: x - m_leaf for every sorted point.
__global__ void k_local_coords(const double *xyz, int64_t n, const int32_t *leaf_cell,
                               const int32_t *leaf_begin, const int32_t *leaf_end, int64_t nleaves,
                               double lo0, double lo1, double lo2, double w, int g, float *loc) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nleaves) return;
  const int cell = leaf_cell[b];
  const int cx = cell % g, cy = (cell / g) % g, cz = cell / (g * g);
  const double m0 = lo0 + (cx + 0.5) * w, m1 = lo1 + (cy + 0.5) * w, m2 = lo2 + (cz + 0.5) * w;
  for (int p = leaf_begin[b]; p < leaf_end[b]; ++p) {
    loc[p] = (float)(xyz[p] - m0);
    loc[n + p] = (float)(xyz[n + p] - m1);
    loc[2 * n + p] = (float)(xyz[2 * n + p] - m2);
  }
}

// ----------------------------------------------------------------- S2M
// One block per (source leaf, direction slot): moments v~_{s,c}[k] =
// sum_{y in s} L_k(y) exp(-i kappa <y - m_s, c>) x_y (Eq. 10, centred
// phases), from the FP64 point coordinates, all in FP64; stored as FP32 (the
// M2L splits them into FP16 pairs; M2M reads them).
template <int O>
__global__ void __launch_bounds__(128) k_s2m_tc(const double *xyz, int64_t n_pts, const int32_t *perm,
                                                const float2 *x, const int32_t *leaf_cell,
                                                const int32_t *leaf_begin, const int32_t *leaf_end, double lo0,
                                                double lo1, double lo2, double w, int g, const double *dir,
                                                double kappa, float *mom, int64_t ncell, int KP, float *maxabs) {
  constexpr int N = O * O * O;
  constexpr int CH = 32;
  constexpr int PER = (N + 127) / 128;
  __shared__ double sl[3][CH][O];
  __shared__ double2 sq[CH];
  const int leaf = blockIdx.x, slot = blockIdx.y;
  const int cell = leaf_cell[leaf];
  const int cx = cell % g, cy = (cell / g) % g, cz = cell / (g * g);
  const double m0 = lo0 + (cx + 0.5) * w, m1 = lo1 + (cy + 0.5) * w, m2 = lo2 + (cz + 0.5) * w;
  const double c0 = dir[3 * slot], c1 = dir[3 * slot + 1], c2 = dir[3 * slot + 2];
  const double inv_h = 2.0 / w;
  double2 acc[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) acc[i] = make_double2(0.0, 0.0);
  const int b = leaf_begin[leaf], e = leaf_end[leaf];
  for (int p0 = b; p0 < e; p0 += CH) {
    const int cnt = min(CH, e - p0);
    if (threadIdx.x < cnt) {
      const int p = p0 + threadIdx.x;
      const double y0 = xyz[p] - m0, y1 = xyz[n_pts + p] - m1, y2 = xyz[2 * n_pts + p] - m2;
      lagrange1d<O>(y0 * inv_h, sl[0][threadIdx.x]);
      lagrange1d<O>(y1 * inv_h, sl[1][threadIdx.x]);
      lagrange1d<O>(y2 * inv_h, sl[2][threadIdx.x]);
      double sn = 0.0, cs = 1.0;
      if (c0 != 0.0 || c1 != 0.0 || c2 != 0.0) sincos(-kappa * (y0 * c0 + y1 * c1 + y2 * c2), &sn, &cs);
      const float2 v = x[perm[p]];
      sq[threadIdx.x] = make_double2(cs * v.x - sn * v.y, cs * v.y + sn * v.x);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int k = threadIdx.x + 128 * i;
      if (k < N) {
        const int kx = k % O, ky = (k / O) % O, kz = k / (O * O);
        for (int q = 0; q < cnt; ++q) {
          const double l = sl[0][q][kx] * sl[1][q][ky] * sl[2][q][kz];
          acc[i].x = fma(l, sq[q].x, acc[i].x);
          acc[i].y = fma(l, sq[q].y, acc[i].y);
        }
      }
    }
    __syncthreads();
  }
  float mx = 0.f;
  float *dst = mom + ((int64_t)slot * ncell + cell) * KP;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int k = threadIdx.x + 128 * i;
    if (k < N) {
      const float re = (float)acc[i].x, im = (float)acc[i].y;
      dst[k] = re;
      dst[N + k] = im;
      mx = fmaxf(mx, fmaxf(abs_or_inf(re), abs_or_inf(im)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) atomic_max_abs(maxabs, mx);
}

// S2M for leaves of at most kSmallLeafS2M points: one warp per (leaf, slot),
// lanes over the n coefficients; the point's 3 o basis values are computed
// once (one lane each) and shared through shared memory; FP64 throughout.
constexpr int kSmallLeafS2M = 16;

template <int O>
__global__ void __launch_bounds__(256) k_s2m_small(const double *xyz, int64_t n_pts, const int32_t *perm,
                                                   const float2 *x, const int32_t *leaf_cell,
                                                   const int32_t *leaf_begin, const int32_t *leaf_end,
                                                   int64_t nleaves, int nslots, double lo0, double lo1, double lo2,
                                                   double w, int g, const double *dir, double kappa, float *mom,
                                                   int64_t ncell, int KP, float *maxabs) {
  constexpr int N = O * O * O;
  constexpr int KPL = (N + 31) / 32;
  __shared__ double sb[8][3 * O + 2];         // per warp: basis values, then the phased x value
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (gw >= nleaves * nslots) return;
  const int64_t leaf = gw / nslots;
  const int slot = (int)(gw - leaf * nslots);
  const int cell = leaf_cell[leaf];
  const int cx = cell % g, cy = (cell / g) % g, cz = cell / (g * g);
  const double m0 = lo0 + (cx + 0.5) * w, m1 = lo1 + (cy + 0.5) * w, m2 = lo2 + (cz + 0.5) * w;
  const double c0 = dir[3 * slot], c1 = dir[3 * slot + 1], c2 = dir[3 * slot + 2];
  const double inv_h = 2.0 / w;
  double ar[KPL], ai[KPL];
#pragma unroll
  for (int j = 0; j < KPL; ++j) ar[j] = ai[j] = 0.0;
  const int b = leaf_begin[leaf], e = leaf_end[leaf];
  for (int p = b; p < e; ++p) {
    const double y0 = xyz[p] - m0, y1 = xyz[n_pts + p] - m1, y2 = xyz[2 * n_pts + p] - m2;
    if (lane < 3 * O) {
      const int ax = lane / O, nu = lane - ax * O;
      const double t = (ax == 0 ? y0 : ax == 1 ? y1 : y2) * inv_h;
      double v = c_lagw[nu];
#pragma unroll
      for (int mu = 0; mu < O; ++mu)
        if (mu != nu) v *= (t - c_cheb[mu]);
      sb[wib][lane] = v;
    } else if (lane == 31) {
      double sn = 0.0, cs = 1.0;
      if (c0 != 0.0 || c1 != 0.0 || c2 != 0.0) sincos(-kappa * (y0 * c0 + y1 * c1 + y2 * c2), &sn, &cs);
      const float2 v = x[perm[p]];
      sb[wib][3 * O] = cs * v.x - sn * v.y;
      sb[wib][3 * O + 1] = cs * v.y + sn * v.x;
    }
    __syncwarp();
    const double qr = sb[wib][3 * O], qi = sb[wib][3 * O + 1];
#pragma unroll
    for (int j = 0; j < KPL; ++j) {
      const int k = lane + 32 * j;
      if (k < N) {
        const double l = sb[wib][k % O] * sb[wib][O + (k / O) % O] * sb[wib][2 * O + k / (O * O)];
        ar[j] = fma(l, qr, ar[j]);
        ai[j] = fma(l, qi, ai[j]);
      }
    }
    __syncwarp();
  }
  float mx = 0.f;
  float *dst = mom + ((int64_t)slot * ncell + cell) * KP;
#pragma unroll
  for (int j = 0; j < KPL; ++j) {
    const int k = lane + 32 * j;
    if (k < N) {
      const float re = (float)ar[j], im = (float)ai[j];
      dst[k] = re;
      dst[N + k] = im;
      mx = fmaxf(mx, fmaxf(abs_or_inf(re), abs_or_inf(im)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0 && mx > 0.f) atomic_max_abs(maxabs, mx);
}

// ------------------------------------------------------ M2M / L2L (FP32)
// Apply E_oct^T (M2M) or E_oct (L2L) axis by axis to the complex smem vector
// (ur, ui) of N = O^3 entries; e1[b][k][l] = L_l((2b - 1 + r_k) / 2).
template <int O>
__device__ void tensor_transfer_f(const float *e1, int oct, bool transpose, float *ur, float *ui, float *tr,
                                  float *ti) {
  constexpr int N = O * O * O;
  const int b[3] = {oct & 1, (oct >> 1) & 1, (oct >> 2) & 1};
  for (int a = 0; a < 3; ++a) {
    const int stride = (a == 0) ? 1 : (a == 1 ? O : O * O);
    const float *m = e1 + b[a] * O * O;
    for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
      const int i = (idx / stride) % O;
      const int base = idx - i * stride;
      float sr = 0.f, si = 0.f;
#pragma unroll
      for (int q = 0; q < O; ++q) {
        const float e = transpose ? m[q * O + i] : m[i * O + q];
        sr = fmaf(e, ur[base + q * stride], sr);
        si = fmaf(e, ui[base + q * stride], si);
      }
      tr[idx] = sr;
      ti[idx] = si;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
      ur[idx] = tr[idx];
      ui[idx] = ti[idx];
    }
    __syncthreads();
  }
}

template <int O>
__global__ void __launch_bounds__(128) k_m2m_f32(const float *cmom, float *pmom, int gp,
                                                 const int32_t *child_slot, const float2 *phase, int nslot_p,
                                                 const float *e1, int KP, float *maxabs) {
  constexpr int N = O * O * O;
  constexpr int PER = (N + 127) / 128;
  __shared__ float ur[N], ui[N], tr[N], ti[N];
  __shared__ float se1[2 * O * O];
  const int64_t cellp = blockIdx.x;
  const int slot = blockIdx.y;
  const int cs = child_slot[slot];
  const int64_t gc = 2 * (int64_t)gp;
  const int64_t ncp = (int64_t)gp * gp * gp, ncc = gc * gc * gc;
  const int x = cellp % gp, y = (cellp / gp) % gp, z = cellp / ((int64_t)gp * gp);
  for (int i = threadIdx.x; i < 2 * O * O; i += blockDim.x) se1[i] = e1[i];
  float ar[PER], ai[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) ar[i] = ai[i] = 0.f;
  __syncthreads();
  for (int oct = 0; oct < 8; ++oct) {
    const int64_t cc = (2 * x + (oct & 1)) + gc * ((2 * y + ((oct >> 1) & 1)) + gc * (2 * z + (oct >> 2)));
    const float *src = cmom + ((int64_t)cs * ncc + cc) * KP;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      float vr = src[k], vi = src[N + k];
      if (phase) {  // times conj(P)
        const float2 p = phase[((int64_t)oct * nslot_p + slot) * N + k];
        const float r = vr * p.x + vi * p.y;
        vi = vi * p.x - vr * p.y;
        vr = r;
      }
      ur[k] = vr;
      ui[k] = vi;
    }
    __syncthreads();
    tensor_transfer_f<O>(se1, oct, true, ur, ui, tr, ti);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int k = threadIdx.x + 128 * i;
      if (k < N) {
        ar[i] += ur[k];
        ai[i] += ui[k];
      }
    }
    __syncthreads();
  }
  float mx = 0.f;
  float *dst = pmom + ((int64_t)slot * ncp + cellp) * KP;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int k = threadIdx.x + 128 * i;
    if (k < N) {
      dst[k] = ar[i];
      dst[N + k] = ai[i];
      mx = fmaxf(mx, fmaxf(abs_or_inf(ar[i]), abs_or_inf(ai[i])));
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) atomic_max_abs(maxabs, mx);
}

template <int O>
__global__ void __launch_bounds__(128) k_l2l_f32(const double *ploc, double *cloc, int gc, const int32_t *pslots,
                                                 const int32_t *pslot_off, const float2 *phase, int nslot_p,
                                                 const float *e1, int KP) {
  constexpr int N = O * O * O;
  constexpr int PER = (N + 127) / 128;
  __shared__ float ur[N], ui[N], tr[N], ti[N];
  __shared__ float se1[2 * O * O];
  const int64_t cellc = blockIdx.x;
  const int cs = blockIdx.y;
  const int gp = gc / 2;
  const int64_t ncp = (int64_t)gp * gp * gp, ncc = (int64_t)gc * gc * gc;
  const int x = cellc % gc, y = (cellc / gc) % gc, z = cellc / ((int64_t)gc * gc);
  const int oct = (x & 1) + 2 * (y & 1) + 4 * (z & 1);
  const int64_t cellp = (x >> 1) + (int64_t)gp * ((y >> 1) + (int64_t)gp * (z >> 1));
  for (int i = threadIdx.x; i < 2 * O * O; i += blockDim.x) se1[i] = e1[i];
  float ar[PER], ai[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) ar[i] = ai[i] = 0.f;
  __syncthreads();
  for (int q = pslot_off[cs]; q < pslot_off[cs + 1]; ++q) {
    const int ps = pslots[q];
    const double *src = ploc + ((int64_t)ps * ncp + cellp) * KP;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      ur[k] = (float)src[k];
      ui[k] = (float)src[KP / 2 + k];
    }
    __syncthreads();
    tensor_transfer_f<O>(se1, oct, false, ur, ui, tr, ti);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int k = threadIdx.x + 128 * i;
      if (k < N) {
        float vr = ur[k], vi = ui[k];
        if (phase) {
          const float2 p = phase[((int64_t)oct * nslot_p + ps) * N + k];
          const float r = vr * p.x - vi * p.y;
          vi = vr * p.y + vi * p.x;
          vr = r;
        }
        ar[i] += vr;
        ai[i] += vi;
      }
    }
    __syncthreads();
  }
  double *dst = cloc + ((int64_t)cs * ncc + cellc) * KP;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int k = threadIdx.x + 128 * i;
    if (k < N) {
      dst[k] += (double)ar[i];
      dst[KP / 2 + k] += (double)ai[i];
    }
  }
}

// ------------------------------------------------ FP32 -> FP16 hi/lo split
// Source: FP32 moments [slot][cell][KP] (cell = x + G y + G^2 z).  Target:
// the parity-split layout the M2L tiles read,
//   [slot][K step of 32][parity (x&1) + 2 (y&1) + 4 (z&1)][z/2][y/2][x/2][32],
// in which the moments of the eight x-neighbours of one parity that a tile
// row needs for one K step are 512 contiguous bytes.
__global__ void k_split(const float *src, int64_t count, int g, int KP, const float *maxabs, int *exp_out,
                        __half *hi, __half *lo, int *err) {
  // scale 2^e with max * 2^e <= 2^14; a level maximum that is not finite, or
  // that the clamped scale cannot bring into FP16's normal range, is a
  // numeric error (error word 2, kept if an earlier error is already there)
  const float mx = *maxabs;
  int e = 0;
  bool bad = !(mx >= 0.f) || isinf(mx);
  if (!bad && mx > 0.f) e = 14 - (int)ceilf(log2f(mx));
  if (e > 60) {
    e = 60;
    bad = bad || ldexpf(mx, e) < 0x1p-14f;
  }
  if (e < -60) {
    e = -60;
    bad = bad || ldexpf(mx, e) > 65504.f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *exp_out = e;
    if (bad) atomicCAS(err, 0, 2);
  }
  const float sc = ldexpf(1.0f, e);
  // one warp per moment row (slot, cell); lane = position in a K step of 32
  const int hg = g >> 1, ksteps = KP >> 5;
  const int64_t ncell = (int64_t)g * g * g, nrows = count / KP;
  const int64_t kstride = (int64_t)8 * hg * hg * hg * 32;   // one K step further
  const int lane = threadIdx.x & 31;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t cell = r % ncell, slot = r / ncell;
    const int x = (int)(cell % g), y = (int)((cell / g) % g), z = (int)(cell / ((int64_t)g * g));
    const int par = (x & 1) + 2 * (y & 1) + 4 * (z & 1);
    const int64_t d0 = (((((slot * ksteps) * 8 + par) * hg + (z >> 1)) * hg + (y >> 1)) * hg + (x >> 1)) * 32 + lane;
    const float *row = src + r * KP;
    for (int kc = 0; kc < ksteps; ++kc) {
      const float v = row[kc * 32 + lane] * sc;
      const __half h = __float2half_rn(v);
      hi[d0 + kc * kstride] = h;
      lo[d0 + kc * kstride] = __float2half_rn(v - __half2float(h));
    }
  }
}

// ------------------------------------------------------------- M2L (TC)
// Arguments of one level's M2L launch.
struct M2lArgs {
  const int32_t *alpha_ops;   // level's op list (global op indices), per alpha
  const int32_t *alpha_off;   // 9 offsets into alpha_ops
  const int32_t *op_off;      // 3 ints per global op
  const int32_t *op_slot;     // slot per global op
  double *loc;                // locals [slot][cell][KP], FP64 sums of FP32 partial sums
  int g;                      // level grid
  int n;                      // nodes per box
  int KP;                     // padded stacked length (= NP)
  const int *mom_exp;         // moment scale exponent of the level (device)
  int op_exp;                 // operator scale exponent of the level
  const int4 *meta;           // per list entry: {op, packed offset, slot, end of its slot run}
  int nsplit;                 // clusters per (tile, alpha), each a contiguous chunk of the op list
  int *err;                   // error word
};

constexpr int kK = 32;                    // K per stage (64-byte rows, two MMA K steps)
constexpr uint32_t kWaitLimit = 1u << 24;

// ------------------------------------------------- M2L (TC, CTA pairs)
// One cluster of two CTAs = 256 targets of parity alpha (an 8 x 4 x 8 block
// of the parent grid; rank 0 the lower z half, rank 1 the upper), one level,
// one chunk of the operator list.  Every MMA is tcgen05.mma.cta_group::2 with
// M = 256 (each CTA's 128 target rows), N = NH = NP / 2 outputs (two passes
// over the list, real then imaginary parts; each CTA holds NH / 2 rows of the
// operator half) and K = 16.  Per K step three products:
//   H  = M_hi O_hi             TMEM columns [0, NH)
//   X += M_lo O_hi + M_hi O_lo TMEM columns [256, 256 + NH)
// so every tensor-core row carries a target and each SM reads half of every
// operator tile.  The tensor core truncates its FP32 accumulator toward zero
// after each instruction, so H lives for one unit of kPU stages (2 kPU
// instructions) only: the MMAs of a unit first build H, then add the unit's
// cross terms to X, and twelve epilogue warps per CTA add H into FP32
// running sums R held in registers while the X instructions run.  X (2^-11
// of H) accumulates over a whole group of operators that share a direction
// slot (at most kPGroupOps); at the group's end X is added to R and R goes to
// the FP64 locals (a transposition through shared memory, then coalesced
// FP64 atomic adds).  Units may span operators of a group (H sums over K and
// over the group's operators alike).
//
// Synchronisation: both CTAs' copies (.cta_group::2 TMA) complete on rank
// 0's full barrier, which rank 0's producer arms with both CTAs' bytes; the
// MMA thread waits there.  Commits multicast to both CTAs (stage free, H
// ready, X ready, all done); the epilogue warps of both CTAs arrive on rank
// 0's H-free / X-free barriers.  Every wait is bounded; a wait that gives up
// sets the error word and the abort flag of both CTAs.
constexpr int kPTM = 128;                  // targets per CTA
constexpr int kPX = 8, kPY = 4, kPZ = 4;   // parent-grid block of one CTA
constexpr int kPU = 3;                     // stages per H unit
constexpr int kPGroupOps = 1 << 20;        // operators per group at most (a whole slot run)
constexpr int kPXUnits = 64;               // units per X accumulation (X drained after them)
// after every second unit one slice of R (32 target rows x 16 columns) goes to
// the locals, so each element of R sums at most 8 (NH / 16) unit drains in FP32
constexpr int kPEpiWarps = 12;             // three per TMEM lane quarter
constexpr int kPEpiWarp0 = 2;              // warps: 0 producer, 1 MMA, 2.. epilogue
constexpr int kPWarps = kPEpiWarp0 + kPEpiWarps;
constexpr int kPThreads = kPWarps * 32;
constexpr int kPEpiThreads = kPEpiWarps * 32;
constexpr uint32_t kPXCol = 256;           // TMEM column of X

template <int NP>
struct PairSmem {
  static constexpr int NH = NP / 2;                // N of one MMA
  static constexpr int NB = NH / 2;                // operator rows one CTA holds
  static constexpr int kRowB = kK * 2;             // 64-byte operand rows
  static constexpr int kM = kPTM * kRowB;          // 128 moment rows
  static constexpr int kO = NB * kRowB;
  static constexpr int kOffMhi = 0, kOffMlo = kM, kOffOhi = 2 * kM, kOffOlo = 2 * kM + kO;
  static constexpr int kStage = 2 * kM + 2 * kO;
  static constexpr int kBuf = 16 * 33 * 4;         // flush: transposition of one 32 x 16 slice
  // at most ~220 KB in all (launches asking for the last few KB of the 227 KB
  // per-CTA limit were refused)
  static constexpr int kStFit = (220 * 1024 - 1024 - kBuf) / kStage;
  static constexpr int kSt = kStFit < 10 ? kStFit : 10;
  static constexpr int kTotal = kSt * kStage + kBuf + 1024;
  static_assert(kStage % 1024 == 0, "stage alignment");
  static_assert(NB % 8 == 0, "operator rows per CTA: whole 8-row swizzle atoms");
  static_assert(kSt >= 2 * kPU + 1, "a unit's stages plus the next unit's must fit");
  static_assert(2 * NB <= 256, "one TMA box per operator share");
};

// Operator image of the pair kernel, rows of 64 B (32 FP16 of K): for each
// (op, output half h, K step of 32, CTA q) a block of 2 NB rows [hi | lo], NB
// rows each, in the 64-byte swizzle the MMA descriptors read; each CTA's share
// of a stage is one TMA box of 2 NB rows (no swizzle in the tensor map: the
// image is already swizzled).
__host__ __device__ __forceinline__ int64_t op_pair_row(int64_t op, int h, int kc, int q, int KSTEPS, int NB) {
  return ((((op * 2 + h) * KSTEPS + kc) * 2 + q) * 2) * NB;
}

__global__ void k_coupling_split_pair(int order, int n, int KP, int NH, const int32_t *op_level,
                                      const int32_t *op_off, const double *op_dir, const double *level_w,
                                      const float *level_scale, double kappa, __half *opk) {
  const int op = blockIdx.x;
  const int row = blockIdx.y;   // 0 .. 2 NH - 1
  const int l = op_level[op];
  const double w = level_w[l], h = 0.5 * w;
  const float sc = level_scale[l];
  const bool im_row = row >= NH;
  const int j = im_row ? row - NH : row;
  const int KSTEPS = KP / 32, NB = NH / 2;
  const int q = j / NB, jj = j - q * NB;
  const double d0 = op_off[3 * op], d1 = op_off[3 * op + 1], d2 = op_off[3 * op + 2];
  const double c0 = op_dir[3 * op], c1 = op_dir[3 * op + 1], c2 = op_dir[3 * op + 2];
  for (int kk = threadIdx.x; kk < KP; kk += blockDim.x) {
    float val = 0.0f;
    const bool kim = kk >= n;
    const int k = kim ? kk - n : kk;
    if (j < n && kk < 2 * n) {
      const int jx = j % order, jy = (j / order) % order, jz = j / (order * order);
      const int kx = k % order, ky = (k / order) % order, kz = k / (order * order);
      const double e0 = h * (c_cheb[jx] - c_cheb[kx]);
      const double e1 = h * (c_cheb[jy] - c_cheb[ky]);
      const double e2 = h * (c_cheb[jz] - c_cheb[kz]);
      const double v0 = w * d0 + e0, v1 = w * d1 + e1, v2 = w * d2 + e2;
      const double r = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
      const double arg = kappa * (r - (e0 * c0 + e1 * c1 + e2 * c2));
      double s, c;
      sincos(arg, &s, &c);
      const double inv = 1.0 / (4.0 * kPi * r);
      const double re = c * inv, im = s * inv;
      double v;   // real-stacked block [[Re, -Im], [Im, Re]]
      if (!im_row) v = kim ? -im : re;
      else v = kim ? re : im;
      val = (float)(v * (double)sc);
    }
    const __half hi = __float2half_rn(val);
    const __half lo = __float2half_rn(val - __half2float(hi));
    const int kc = kk >> 5, e = kk & 31, hh = im_row ? 1 : 0;
    const int chunk = (e >> 3) ^ ((jj >> 1) & 3);
    const int64_t base = op_pair_row(op, hh, kc, q, KSTEPS, NB) * 32 + (int64_t)jj * 32 + chunk * 8 + (e & 7);
    opk[base] = hi;
    opk[base + (int64_t)NB * 32] = lo;
  }
}

template <int NP>
__global__ void __cluster_dims__(2, 1, 1) __maxnreg__(128)
    k_m2l_pair(const __grid_constant__ CUtensorMap map_mhi, const __grid_constant__ CUtensorMap map_mlo,
               const __grid_constant__ CUtensorMap map_op, const M2lArgs args) {
  using S = PairSmem<NP>;
  constexpr int NH = S::NH;
  constexpr int NB = S::NB;
  constexpr int KSTEPS = NP / kK;      // stages per operator and half
  constexpr int NCH = NH / 16;         // 16-column chunks of one half
  constexpr int MAXC = (NCH + 2) / 3;  // chunks per epilogue warp at most
  constexpr int kSt = S::kSt;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float *buf = reinterpret_cast<float *>(smem + kSt * S::kStage);   // [16][kPBufRS]
  constexpr int kGo = kSt + 2;         // ring of per-unit "go" barriers
  __shared__ uint64_t go_bar[kGo], empty_bar[kSt], h_full, x_full, x_empty, fin_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;

  const uint32_t rank = ptx::cluster_rank();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = args.g, gp = g >> 1;
  const int tiles_x = (gp + kPX - 1) / kPX, tiles_y = (gp + kPY - 1) / kPY;
  const int pt = blockIdx.x >> 1;
  const int X0 = (pt % tiles_x) * kPX;
  const int Y0 = ((pt / tiles_x) % tiles_y) * kPY;
  const int Z0 = (pt / (tiles_x * tiles_y)) * (2 * kPZ) + (int)rank * kPZ;
  const int alpha = blockIdx.y;
  const int ax = alpha & 1, ay = (alpha >> 1) & 1, az = (alpha >> 2) & 1;
  const int a0 = args.alpha_off[alpha], na = args.alpha_off[alpha + 1] - a0;
  const int i0 = a0 + (int)(((int64_t)na * blockIdx.z) / args.nsplit);
  const int i1 = a0 + (int)(((int64_t)na * (blockIdx.z + 1)) / args.nsplit);

  if (tid == 0) {
    for (int s = 0; s < kSt; ++s) ptx::mbar_init(&empty_bar[s], 1);
    // a unit may start once its stages have landed (rank 0's producer arms
    // the barrier with both CTAs' bytes) and H is free (every epilogue warp
    // of both CTAs arrives after draining the previous unit)
    for (int b = 0; b < kGo; ++b) ptx::mbar_init(&go_bar[b], 1 + 2 * kPEpiWarps);
    ptx::mbar_init(&h_full, 1);
    ptx::mbar_init(&x_full, 1);
    ptx::mbar_init(&fin_bar, 1);
    ptx::mbar_init(&x_empty, 2 * kPEpiWarps);
    s_abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc_pair(&tmem_base, 512);
    ptx::tmem_relinquish_pair();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t peer_abort = ptx::cluster_addr(&s_abort, rank ^ 1u);
  auto abort_both = [&]() {
    atomicExch(args.err, 1);
    s_abort = 1;
    ptx::st_cluster_u32(peer_abort, 1u);
  };
  auto group_end = [&](int ii) { return min(args.meta[ii].w, min(ii + kPGroupOps, i1)); };

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------ producer (both CTAs)
      ptx::prefetch_tensormap(&map_mhi);
      ptx::prefetch_tensormap(&map_mlo);
      ptx::prefetch_tensormap(&map_op);
      const uint32_t go0 = ptx::cluster_addr(&go_bar[0], 0);
      uint32_t it = 0, un = 0;
      bool ok = true;
      for (int h = 0; h < 2 && ok; ++h) {
        for (int ii = i0; ii < i1 && ok;) {
          const int jj = group_end(ii);
          const int ns = (jj - ii) * KSTEPS;
          int sg = 0;                        // stage within the group
          int4 nxt = args.meta[ii];
          for (int oi = ii; oi < jj && ok; ++oi) {
            const int4 m = nxt;
            if (oi + 1 < jj) nxt = args.meta[oi + 1];   // next entry's metadata in flight
            const int op = m.x, slot = m.z;
            // sources t - d of this tile: parity (alpha - d) & 1 per axis,
            // and in that parity's half grid the tile's block shifted by
            // (alpha - d - parity) / 2
            const int sx = ax - ((m.y & 255) - 128), sy = ay - (((m.y >> 8) & 255) - 128),
                      sz = az - (((m.y >> 16) & 255) - 128);
            const int px = sx & 1, py = sy & 1, pz = sz & 1;
            const int x0 = X0 + (sx - px) / 2, y0 = Y0 + (sy - py) / 2, z0 = Z0 + (sz - pz) / 2;
            const int qbase = (slot * KSTEPS) * 8 + px + 2 * py + 4 * pz;
            for (int kc = 0; kc < KSTEPS; ++kc, ++it, ++sg) {
              if (sg % kPU == 0) {           // a unit starts: arm its go barrier
                if (rank == 0) ptx::mbar_expect_tx(&go_bar[un % kGo], min(kPU, ns - sg) * 2 * S::kStage);
                ++un;
              }
              const int st = it % kSt;
              const uint32_t ph = (it / kSt) & 1;
              if (!ptx::mbar_wait(&empty_bar[st], ph ^ 1, kWaitLimit)) { ok = false; break; }
              uint8_t *base = smem + st * S::kStage;
              const uint32_t gb = go0 + 8u * ((un - 1) % kGo);
              ptx::tma_load_5d_pair(base + S::kOffMhi, &map_mhi, gb, 0, x0, y0, z0, qbase + kc * 8);
              ptx::tma_load_5d_pair(base + S::kOffMlo, &map_mlo, gb, 0, x0, y0, z0, qbase + kc * 8);
              ptx::tma_load_2d_pair(base + S::kOffOhi, &map_op, gb, 0,
                                    (int)(op_pair_row(op, h, kc, (int)rank, KSTEPS, NB) / 8));
            }
          }
          ii = jj;
        }
      }
      // copies of both CTAs still in flight land before the pair leaves: the
      // last unit's barrier completes only after all of them (rank 0 counts
      // both CTAs' bytes; already complete on a normal run)
      if (rank == 0 && un > 0 && ok && !ptx::mbar_wait(&go_bar[(un - 1) % kGo], ((un - 1) / kGo) & 1, kWaitLimit))
        ok = false;
      if (!ok) abort_both();
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      // ------------------------------------------------ MMA issuer (rank 0)
      constexpr uint32_t idesc = ptx::idesc_f16_f32(256, NH);
      uint32_t it = 0, hu = 0, xg = 0;
      bool ok = true;
      for (int h = 0; h < 2 && ok; ++h) {
        for (int ii = i0; ii < i1 && ok;) {
          const int jj = group_end(ii);
          const int ns = (jj - ii) * KSTEPS;
          for (int u0 = 0, gu = 0; u0 < ns && ok; u0 += kPU, ++gu) {
            const int nst = min(kPU, ns - u0);
            const bool x_first = (gu % kPXUnits) == 0;
            const bool x_last = (gu % kPXUnits) == kPXUnits - 1 || u0 + kPU >= ns;
            // one wait per unit: its stages landed and H is free
            if (!ptx::mbar_wait(&go_bar[hu % kGo], (hu / kGo) & 1, kWaitLimit)) { ok = false; break; }
            ptx::tc_fence_after();
            for (int t = 0; t < nst; ++t) {
              const uint32_t base = ptx::smem_u32(smem + ((it + t) % kSt) * S::kStage);
#pragma unroll
              for (int j = 0; j < 2; ++j) {
                const uint32_t o = 32u * j;
                ptx::mma_f16_pair(tmem, ptx::sdesc_k_sw64(base + S::kOffMhi + o),
                                  ptx::sdesc_k_sw64(base + S::kOffOhi + o), idesc, (t | j) ? 1u : 0u);
              }
            }
            ptx::mma_commit_pair(&h_full);
            if (x_first && xg > 0) {
              if (!ptx::mbar_wait(&x_empty, (xg - 1) & 1, kWaitLimit)) { ok = false; break; }
              ptx::tc_fence_after();
            }
            for (int t = 0; t < nst; ++t) {
              const int st = (it + t) % kSt;
              const uint32_t base = ptx::smem_u32(smem + st * S::kStage);
#pragma unroll
              for (int j = 0; j < 2; ++j) {
                const uint32_t o = 32u * j;
                ptx::mma_f16_pair(tmem + kPXCol, ptx::sdesc_k_sw64(base + S::kOffMlo + o),
                                  ptx::sdesc_k_sw64(base + S::kOffOhi + o), idesc,
                                  (x_first && t == 0 && j == 0) ? 0u : 1u);
                ptx::mma_f16_pair(tmem + kPXCol, ptx::sdesc_k_sw64(base + S::kOffMhi + o),
                                  ptx::sdesc_k_sw64(base + S::kOffOlo + o), idesc, 1u);
              }
              ptx::mma_commit_pair(&empty_bar[st]);
            }
            if (x_last) {
              ptx::mma_commit_pair(&x_full);
              ++xg;
            }
            it += nst;
            ++hu;
          }
          if (!ok) break;
          ii = jj;
        }
      }
      if (!ok) abort_both();
      // every MMA has finished with shared memory and TMEM of both CTAs
      ptx::mma_commit_pair(&fin_bar);
    }
  } else {
    // ------------------------------------------------ epilogue (both CTAs)
    const int e = warp - kPEpiWarp0;          // 0..11
    const int q = warp & 3;                   // TMEM lane quarter this warp may read
    const int wq = e >> 2;                    // column third of H / X
    const int c_lo = (NCH * wq) / 3, nc = (NCH * (wq + 1)) / 3 - c_lo;
    const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
    const uint32_t go0 = ptx::cluster_addr(&go_bar[0], 0);
    const uint32_t x_empty0 = ptx::cluster_addr(&x_empty, 0);
    const int64_t ncell = (int64_t)g * g * g;
    const int n = args.n;
    const double inv = (double)ldexpf(1.0f, -(args.op_exp + *args.mom_exp));
    const int te = tid - kPEpiWarp0 * 32;     // 0..383
    float R[MAXC * 16];
#pragma unroll
    for (int i = 0; i < MAXC * 16; ++i) R[i] = 0.f;
    uint32_t hu = 0, xg = 0;
    bool bad = false;
    if (lane == 0) ptx::mbar_arrive_cluster(go0);   // H is free for unit 0
    // bounded wait that also gives up once the other warps or CTA aborted;
    // the wall clock is read only after 256 failed tries
    auto wait_local = [&](uint64_t *bar, uint32_t ph) {
      uint64_t t0 = 0;
      for (uint32_t t = 0; t < kWaitLimit; ++t) {
        if (ptx::mbar_try_wait(bar, ph)) return true;
        if ((t & 255) == 255) {
          if (*(volatile int *)&s_abort) return false;
          const uint64_t now = ptx::global_ns();
          if (t0 == 0) t0 = now;
          else if (now - t0 > 1000000000ull) return false;
        }
      }
      return false;
    };
    // add the region at TMEM column `col0` to R
    auto drain = [&](uint32_t col0) {
#pragma unroll
      for (int c = 0; c < MAXC; ++c) {
        if (c < nc) {
          float v[16];
          ptx::tmem_ld16(tmem + lane_addr + col0 + (uint32_t)((c_lo + c) * 16), v);
          ptx::tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 16; ++i) R[c * 16 + i] += v[i];
        }
      }
    };
    // slice (chunk k, lane quarter qs) of R -> locals: its one owner warp
    // transposes the 32 x 16 values through shared memory, then every
    // epilogue thread adds a part with FP64 atomics (consecutive lanes:
    // consecutive columns of one target row).  Columns at or beyond n hold
    // exact zeros (the operator rows there are zero) and are skipped.
    // Returns the common decision to stop, taken at the first barrier.
    auto flush_slice = [&](int k, int qs, int slot, int h) {
      if (q == qs) {
#pragma unroll
        for (int c = 0; c < MAXC; ++c) {
          if (c < nc && c_lo + c == k) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              buf[i * 33 + lane] = R[c * 16 + i];
              R[c * 16 + i] = 0.f;
            }
          }
        }
      }
      if (ptx::named_bar_or(1, kPEpiThreads, bad || *(volatile int *)&s_abort)) return true;
      for (int idx = te; idx < 32 * 16; idx += kPEpiThreads) {
        const int rr = qs * 32 + (idx >> 4), cc = idx & 15;
        const int col = k * 16 + cc;
        const int XX = X0 + (rr & 7), YY = Y0 + ((rr >> 3) & 3), ZZ = Z0 + (rr >> 5);
        if (col < n && XX < gp && YY < gp && ZZ < gp) {
          const int64_t cl = (2 * XX + ax) + (int64_t)g * ((2 * YY + ay) + (int64_t)g * (2 * ZZ + az));
          atomicAdd(args.loc + ((int64_t)slot * ncell + cl) * args.KP + h * (args.KP / 2) + col,
                    (double)buf[cc * 33 + (idx >> 4)] * inv);
        }
      }
      ptx::named_bar(1, kPEpiThreads);
      return false;
    };
    bool stop = false;
    for (int h = 0; h < 2 && !stop; ++h) {
      for (int ii = i0; ii < i1 && !stop;) {
        const int jj = group_end(ii);
        const int slot = args.meta[ii].z;
        const int ns = (jj - ii) * KSTEPS;
        int roll = 0;                     // next slice of the rolling flush: chunk roll / 4, quarter roll % 4
        for (int u0 = 0, gu = 0; u0 < ns && !stop; u0 += kPU, ++gu) {
          const bool x_last = (gu % kPXUnits) == kPXUnits - 1 || u0 + kPU >= ns;
          if (!bad && !wait_local(&h_full, hu & 1)) bad = true;
          ++hu;
          if (!bad) {
            ptx::tc_fence_after();
            drain(0);
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive_cluster(go0 + 8u * (hu % kGo));   // H free for unit hu
          }
          if (x_last) {
            if (!bad && !wait_local(&x_full, xg & 1)) bad = true;
            ++xg;
            if (!bad) {
              ptx::tc_fence_after();
              drain(kPXCol);
              ptx::tc_fence_before();
              __syncwarp();
              if (lane == 0) ptx::mbar_arrive_cluster(x_empty0);
            }
          }
          if (u0 + kPU >= ns) {
            // the group's slot (or output half) changes next: everything in R
            // goes out; one decision for all epilogue warps before the barriers
            for (int k = 0; k < NCH && !stop; ++k)
              for (int qs = 0; qs < 4 && !stop; ++qs) stop = flush_slice(k, qs, slot, h);
            if (stop) break;
          } else if (gu & 1) {
            stop = flush_slice(roll >> 2, roll & 3, slot, h);
            roll = (roll + 1) % (4 * NCH);
          }
        }
        ii = jj;
      }
    }
    if (bad) abort_both();
  }
  // ------------------------------------------------ teardown (both CTAs)
  if (warp == 1 && lane == 0) {
    // the last commit of rank 0's MMA thread reached this CTA
    if (!ptx::mbar_wait(&fin_bar, 0, kWaitLimit)) atomicExch(args.err, 1);
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();
  ptx::tc_fence_after();
  if (warp == 1) ptx::tmem_dealloc_pair(tmem, 512);
}

template <int O>
__device__ __forceinline__ double pick(const double *a, int i) {
  double v = a[0];
#pragma unroll
  for (int j = 1; j < O; ++j) v = (i == j) ? a[j] : v;
  return v;
}

// ----------------------------------------------------------------- L2T
// y_x = sum_c exp(i kappa <x - m_t, c>) sum_k L_k(x) g~_{t,c}[k] (Eq. 14,
// centred phases), from the FP64 point coordinates and the FP64 locals, all in
// FP64.  Leaves of more than kSmallLeaf points: one block per leaf, one
// thread per target point, the leaf's coefficients of one slot staged in
// shared memory (broadcast reads).
template <int O>
__global__ void __launch_bounds__(128) k_l2t_tc(const double *xyz, int64_t n_pts, const int32_t *leaf_cell,
                                                const int32_t *leaf_begin, const int32_t *leaf_end, double lo0,
                                                double lo1, double lo2, double w, int g, const double *dir,
                                                int nslots, double kappa, const double *loc, int64_t ncell, int KP,
                                                float2 *ysorted) {
  constexpr int N = O * O * O;
  __shared__ double gs[2 * N];
  const int leaf = blockIdx.x;
  const int cell = leaf_cell[leaf];
  const int cx = cell % g, cy = (cell / g) % g, cz = cell / (g * g);
  const double m0 = lo0 + (cx + 0.5) * w, m1 = lo1 + (cy + 0.5) * w, m2 = lo2 + (cz + 0.5) * w;
  const double inv_h = 2.0 / w;
  const int b = leaf_begin[leaf], e = leaf_end[leaf];
  for (int p0 = b; p0 < e; p0 += blockDim.x) {
    const int p = p0 + threadIdx.x;
    const bool act = p < e;
    double y0 = 0.0, y1 = 0.0, y2 = 0.0;
    if (act) {
      y0 = xyz[p] - m0;
      y1 = xyz[n_pts + p] - m1;
      y2 = xyz[2 * n_pts + p] - m2;
    }
    double lx[O], ly[O], lz[O];
    lagrange1d<O>(y0 * inv_h, lx);
    lagrange1d<O>(y1 * inv_h, ly);
    lagrange1d<O>(y2 * inv_h, lz);
    double tx = 0.0, ty = 0.0;
    for (int slot = 0; slot < nslots; ++slot) {
      const double *src = loc + ((int64_t)slot * ncell + cell) * KP;
      __syncthreads();
      for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) gs[i] = src[i < N ? i : KP / 2 + (i - N)];
      __syncthreads();
      double re = 0.0, im = 0.0;
#pragma unroll 1
      for (int kz = 0; kz < O; ++kz) {
#pragma unroll
        for (int ky = 0; ky < O; ++ky) {
          const double lyz = ly[ky] * pick<O>(lz, kz);
          const int k0 = O * (ky + O * kz);
#pragma unroll
          for (int kx = 0; kx < O; ++kx) {
            const double l = lx[kx] * lyz;
            re = fma(l, gs[k0 + kx], re);
            im = fma(l, gs[N + k0 + kx], im);
          }
        }
      }
      const double c0 = dir[3 * slot], c1 = dir[3 * slot + 1], c2 = dir[3 * slot + 2];
      if (c0 == 0.0 && c1 == 0.0 && c2 == 0.0) {
        tx += re;
        ty += im;
      } else {
        double sn, cs;
        sincos(kappa * (y0 * c0 + y1 * c1 + y2 * c2), &sn, &cs);
        tx += re * cs - im * sn;
        ty += re * sn + im * cs;
      }
    }
    if (act) ysorted[p] = make_float2((float)tx, (float)ty);
  }
}

// Leaves of at most kSmallLeaf points (uniform trees: ~2 points a leaf): one
// warp per leaf, lanes over the n coefficients of one point at a time,
// partial sums reduced across the warp; all in FP64.

template <int O>
__global__ void __launch_bounds__(256) k_l2t_small(const double *xyz, int64_t n_pts, const int32_t *leaf_cell,
                                                   const int32_t *leaf_begin, const int32_t *leaf_end,
                                                   int64_t nleaves, double lo0, double lo1, double lo2, double w,
                                                   int g, const double *dir, int nslots, double kappa,
                                                   const double *loc, int64_t ncell, int KP, float2 *ysorted) {
  constexpr int N = O * O * O;
  constexpr int KPL = (N + 31) / 32;
  __shared__ double sb[8][3 * O];             // per warp: the point's 1-D basis values
  const int64_t leaf = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (leaf >= nleaves) return;
  const int cell = leaf_cell[leaf];
  const int cx = cell % g, cy = (cell / g) % g, cz = cell / (g * g);
  const double m[3] = {lo0 + (cx + 0.5) * w, lo1 + (cy + 0.5) * w, lo2 + (cz + 0.5) * w};
  const double inv_h = 2.0 / w;
  const int b = leaf_begin[leaf], e = leaf_end[leaf];
  for (int p = b; p < e; ++p) {
    const double y0 = xyz[p] - m[0], y1 = xyz[n_pts + p] - m[1], y2 = xyz[2 * n_pts + p] - m[2];
    // lane a * O + nu computes L_nu along axis a (one FP64 product chain per lane)
    if (lane < 3 * O) {
      const int ax = lane / O, nu = lane - ax * O;
      const double t = (ax == 0 ? y0 : ax == 1 ? y1 : y2) * inv_h;
      double v = c_lagw[nu];
#pragma unroll
      for (int mu = 0; mu < O; ++mu)
        if (mu != nu) v *= (t - c_cheb[mu]);
      sb[wib][lane] = v;
    }
    __syncwarp();
    double l[KPL];
#pragma unroll
    for (int j = 0; j < KPL; ++j) {
      const int k = lane + 32 * j;
      l[j] = (k < N) ? sb[wib][k % O] * sb[wib][O + (k / O) % O] * sb[wib][2 * O + k / (O * O)] : 0.0;
    }
    __syncwarp();
    double tx = 0.0, ty = 0.0;
    for (int slot = 0; slot < nslots; ++slot) {
      const double *src = loc + ((int64_t)slot * ncell + cell) * KP;
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int j = 0; j < KPL; ++j) {
        const int k = lane + 32 * j;
        if (k < N) {
          re = fma(l[j], src[k], re);
          im = fma(l[j], src[KP / 2 + k], im);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      const double c0 = dir[3 * slot], c1 = dir[3 * slot + 1], c2 = dir[3 * slot + 2];
      if (c0 == 0.0 && c1 == 0.0 && c2 == 0.0) {
        tx += re;
        ty += im;
      } else {
        double sn, cs;
        sincos(kappa * (y0 * c0 + y1 * c1 + y2 * c2), &sn, &cs);
        tx += re * cs - im * sn;
        ty += re * sn + im * cs;
      }
    }
    if (lane == 0) ysorted[p] = make_float2((float)tx, (float)ty);
  }
}

// ----------------------------------------------------- nearfield (FP32)
// exp(i 2 pi t) for t = kappa r / (2 pi) >= 0.  t is reduced to f = t - rint(t)
// in [-1/2, 1/2]: adding and removing 1.5 * 2^23 rounds to the nearest integer
// for t < 2^22, and t - rint(t) is exact (Sterbenz).  The hardware sine and
// cosine then take 2 pi f in [-pi, pi], where CUDA documents their absolute
// error as below 2^-21.4 (sine) and 2^-21.1 (cosine).
__device__ __forceinline__ void exp_i_rev(float t, float &sn, float &cs) {
  const float n = __fadd_rn(__fadd_rn(t, 12582912.f), -12582912.f);
  __sincosf(6.28318530717958647692f * (t - n), &sn, &cs);
}

constexpr int kP2pT = 4;   // targets per thread of k_p2p_f32

// Staged sources (k, k + 1) for k = 0, 2, .. < cnt2 against the thread's
// kP2pT targets, two sources per packed FP32 instruction: adds
// x_y exp(i kappa r) / (4 pi r) into the packed sums (even, odd source)
// cr / ci.  Per pair: the differences, r^2, 1 / r (hardware rsqrt), kappa r
// in revolutions t = kap_rev r, its exact reduction f = t - rint(t) (adding and
// removing 1.5 * 2^23 rounds to the nearest integer for t < 2^22; t - rint(t)
// is exact), the hardware sine and cosine of 2 pi f in [-pi, pi], and the
// complex multiply-add.  SELF (the target's own leaf): coincident points
// (the zero diagonal) add 0.  Other leaves hold no point equal to the target
// (equal coordinates share a leaf); there r^2 gets 2^-100 added, which
// leaves every representable distance unchanged and keeps 1 / r finite for
// two distinct points that round to the same FP32 coordinates.
template <bool SELF>
__device__ __forceinline__ void p2p_staged(const float *qx, const float *qy, const float *qz, const float *vx,
                                           const float *vy, const float *nvy, int cnt2,
                                           const uint64_t (&PX)[kP2pT], const uint64_t (&PY)[kP2pT],
                                           const uint64_t (&PZ)[kP2pT], uint64_t (&CR)[kP2pT],
                                           uint64_t (&CI)[kP2pT], uint64_t KAP) {
  const uint64_t MAG = ptx::f2_pack(12582912.f, 12582912.f);
  const uint64_t TWOPI = ptx::f2_pack(6.28318530717958647692f, 6.28318530717958647692f);
  const uint64_t TINY = ptx::f2_pack(0x1p-100f, 0x1p-100f);
  for (int k = 0; k < cnt2; k += 2) {
    const uint64_t QX = *reinterpret_cast<const uint64_t *>(qx + k);
    const uint64_t QY = *reinterpret_cast<const uint64_t *>(qy + k);
    const uint64_t QZ = *reinterpret_cast<const uint64_t *>(qz + k);
    const uint64_t VX = *reinterpret_cast<const uint64_t *>(vx + k);
    const uint64_t VY = *reinterpret_cast<const uint64_t *>(vy + k);
    const uint64_t NVY = *reinterpret_cast<const uint64_t *>(nvy + k);
#pragma unroll
    for (int u = 0; u < kP2pT; ++u) {
      const uint64_t D0 = ptx::f2_sub(PX[u], QX), D1 = ptx::f2_sub(PY[u], QY), D2 = ptx::f2_sub(PZ[u], QZ);
      uint64_t R2 = ptx::f2_fma(D0, D0, ptx::f2_fma(D1, D1, ptx::f2_mul(D2, D2)));
      if (!SELF) R2 = ptx::f2_add(R2, TINY);
      float r2a, r2b;
      ptx::f2_unpack(R2, r2a, r2b);
      float ira = ptx::rsqrt_approx(r2a), irb = ptx::rsqrt_approx(r2b);
      if (SELF) {
        ira = r2a > 0.f ? ira : 0.f;
        irb = r2b > 0.f ? irb : 0.f;
      }
      const uint64_t IR = ptx::f2_pack(ira, irb);
      const uint64_t T = ptx::f2_mul(ptx::f2_mul(R2, IR), KAP);
      const uint64_t N = ptx::f2_sub(ptx::f2_add(T, MAG), MAG);
      const uint64_t TH = ptx::f2_mul(ptx::f2_sub(T, N), TWOPI);
      float ta, tb, sa, ca, sb, cb;
      ptx::f2_unpack(TH, ta, tb);
      __sincosf(ta, &sa, &ca);
      __sincosf(tb, &sb, &cb);
      const uint64_t A = ptx::f2_mul(IR, ptx::f2_pack(ca, cb)), B = ptx::f2_mul(IR, ptx::f2_pack(sa, sb));
      CR[u] = ptx::f2_fma(B, NVY, ptx::f2_fma(A, VX, CR[u]));
      CI[u] = ptx::f2_fma(B, VX, ptx::f2_fma(A, VY, CI[u]));
    }
  }
}

// Nearfield, leaves above kSmallLeaf points.  Blocks (target leaf, target
// chunk): blockIdx.y of gridDim.y chunks of kP2pT x blockDim.x targets of the
// leaf (a leaf of 512 points gives 128-thread blocks one chunk, 32-thread
// blocks four, so that few large leaves still fill the SMs).  Each thread
// owns up to kP2pT targets of its chunk (strided by the block size); the
// source points of every nearfield leaf are staged through shared memory,
// blockDim.x at a time, and p2p_staged runs them against the thread's
// targets.  Positions are leaf-local FP32 (m_t - m_s = w d is exact), so
// |x - y| keeps FP32 relative accuracy.  Every 128 sources the FP32 partial
// sums are added to FP64 totals, so long source lists (512-point leaves) do
// not accumulate FP32 rounding.  blockDim.x divides 128.
__global__ void __launch_bounds__(128, 8) k_p2p_f32(const float *tl, int64_t nt, const int32_t *tperm,
                                                 const int32_t *leaf_cell, const int32_t *leaf_begin,
                                                 const int32_t *leaf_end, const float *sl, int64_t ns,
                                                 const int32_t *sperm, const int32_t *s_leaf_of_cell,
                                                 const int32_t *sb, const int32_t *se, int g, float w,
                                                 const int32_t *near_off, int nnear, float kappa,
                                                 const float2 *x, const float2 *ysorted, float2 *y) {
  // staged sources, one array per component (pairs of consecutive sources
  // are one 8-byte load); the odd slot after an odd count holds a zero value
  __shared__ __align__(16) float qx[128], qy[128], qz[128], vx[128], vy[128], nvy[128];
  // FP64 totals of the thread's targets (shared memory keeps them out of the
  // registers of the inner loop: 64 registers, eight blocks per SM)
  __shared__ double acc_r[kP2pT][128], acc_i[kP2pT][128];
  const int leaf = blockIdx.x;
  const int cell = leaf_cell[leaf];
  const int cx = cell % g, cy = (cell / g) % g, cz = cell / (g * g);
  const int b = leaf_begin[leaf], e = leaf_end[leaf];
  const float inv4pi = (float)(1.0 / (4.0 * kPi));
  const float kap_rev = (float)((double)kappa / (2.0 * kPi));   // kappa r in revolutions
  const uint64_t KAP = ptx::f2_pack(kap_rev, kap_rev);
  for (int p0 = b + blockIdx.y * kP2pT * blockDim.x; p0 < e; p0 += gridDim.y * kP2pT * blockDim.x) {
    uint64_t PX[kP2pT], PY[kP2pT], PZ[kP2pT];
#pragma unroll
    for (int u = 0; u < kP2pT; ++u) {
      const int p = p0 + u * blockDim.x + threadIdx.x;
      const bool act = p < e;
      const float px = act ? tl[p] : 0.f, py = act ? tl[nt + p] : 0.f, pz = act ? tl[2 * nt + p] : 0.f;
      PX[u] = ptx::f2_pack(px, px);
      PY[u] = ptx::f2_pack(py, py);
      PZ[u] = ptx::f2_pack(pz, pz);
      acc_r[u][threadIdx.x] = 0.0;
      acc_i[u][threadIdx.x] = 0.0;
    }
    for (int i = 0; i < nnear; ++i) {
      const int dx = near_off[3 * i], dy = near_off[3 * i + 1], dz = near_off[3 * i + 2];
      const int sx = cx - dx, sy = cy - dy, sz = cz - dz;
      if (sx < 0 || sy < 0 || sz < 0 || sx >= g || sy >= g || sz >= g) continue;
      const int s = s_leaf_of_cell[sx + g * (sy + g * sz)];
      if (s < 0) continue;
      const bool self = (dx | dy | dz) == 0;
      const float ox = w * dx, oy = w * dy, oz = w * dz;   // m_t - m_s
      uint64_t CR[kP2pT], CI[kP2pT];
#pragma unroll
      for (int u = 0; u < kP2pT; ++u) CR[u] = CI[u] = 0ull;   // (+0, +0)
      for (int q0 = sb[s]; q0 < se[s]; q0 += blockDim.x) {   // chunks of one source per thread
        const int cnt = min((int)blockDim.x, se[s] - q0);
        __syncthreads();
        if (threadIdx.x < cnt) {
          const int q = q0 + threadIdx.x;
          // source position relative to the target leaf's centre, x_y / (4 pi)
          qx[threadIdx.x] = sl[q] - ox;
          qy[threadIdx.x] = sl[ns + q] - oy;
          qz[threadIdx.x] = sl[2 * ns + q] - oz;
          const float2 v = x[sperm[q]];
          vx[threadIdx.x] = v.x * inv4pi;
          vy[threadIdx.x] = v.y * inv4pi;
          nvy[threadIdx.x] = -v.y * inv4pi;
        } else if (threadIdx.x == cnt) {   // odd count: a source of value 0
          qx[threadIdx.x] = qy[threadIdx.x] = qz[threadIdx.x] = 0.f;
          vx[threadIdx.x] = vy[threadIdx.x] = nvy[threadIdx.x] = 0.f;
        }
        __syncthreads();
        const int cnt2 = (cnt + 1) & ~1;
        if (self)
          p2p_staged<true>(qx, qy, qz, vx, vy, nvy, cnt2, PX, PY, PZ, CR, CI, KAP);
        else
          p2p_staged<false>(qx, qy, qz, vx, vy, nvy, cnt2, PX, PY, PZ, CR, CI, KAP);
        if (((q0 - sb[s]) & 127) + (int)blockDim.x >= 128 || q0 + (int)blockDim.x >= se[s]) {
#pragma unroll
          for (int u = 0; u < kP2pT; ++u) {
            float r0, r1, i0, i1;
            ptx::f2_unpack(CR[u], r0, r1);
            ptx::f2_unpack(CI[u], i0, i1);
            acc_r[u][threadIdx.x] += (double)r0 + (double)r1;
            acc_i[u][threadIdx.x] += (double)i0 + (double)i1;
            CR[u] = CI[u] = 0ull;
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kP2pT; ++u) {
      const int p = p0 + u * blockDim.x + threadIdx.x;
      if (p < e) {
        const float2 f = ysorted[p];
        y[tperm[p]] = make_float2((float)(acc_r[u][threadIdx.x] + (double)f.x),
                                  (float)(acc_i[u][threadIdx.x] + (double)f.y));
      }
    }
  }
}

// Nearfield for several right-hand sides (leaves above kSmallLeaf points):
// one block per target leaf, one thread per target point (strided), and per
// pass kP2pRG right-hand sides: each pair's kernel value f(x, y) is formed
// once and multiplied into every right-hand side of the pass, two sources per
// packed FP32 instruction.  Sources (positions and the pass's x values) are
// staged through shared memory in chunks of the block size; chunk sums in
// FP32 are added into FP64.
constexpr int kP2pRG = 8;

// Staged sources (k, k + 1), k = 0, 2, .. < cnt2, against the thread's
// target for kP2pRG right-hand sides: the kernel value f(x, y) (same steps as
// p2p_staged) is formed once per pair, two sources per packed instruction,
// and multiplied into every right-hand side.  sv4[r][k / 2] holds
// {vx_k, vx_k+1, vy_k, vy_k+1} of right-hand side r (x_y / (4 pi)).
template <bool SELF>
__device__ __forceinline__ void p2p_staged_mrhs(const float *qx, const float *qy, const float *qz,
                                                const float4 (*sv4)[64], int cnt2, uint64_t PX, uint64_t PY,
                                                uint64_t PZ, uint64_t (&CR)[kP2pRG], uint64_t (&CI)[kP2pRG],
                                                uint64_t KAP) {
  const uint64_t MAG = ptx::f2_pack(12582912.f, 12582912.f);
  const uint64_t TWOPI = ptx::f2_pack(6.28318530717958647692f, 6.28318530717958647692f);
  const uint64_t TINY = ptx::f2_pack(0x1p-100f, 0x1p-100f);
  for (int k = 0; k < cnt2; k += 2) {
    const uint64_t D0 = ptx::f2_sub(PX, *reinterpret_cast<const uint64_t *>(qx + k));
    const uint64_t D1 = ptx::f2_sub(PY, *reinterpret_cast<const uint64_t *>(qy + k));
    const uint64_t D2 = ptx::f2_sub(PZ, *reinterpret_cast<const uint64_t *>(qz + k));
    uint64_t R2 = ptx::f2_fma(D0, D0, ptx::f2_fma(D1, D1, ptx::f2_mul(D2, D2)));
    if (!SELF) R2 = ptx::f2_add(R2, TINY);
    float r2a, r2b;
    ptx::f2_unpack(R2, r2a, r2b);
    float ira = ptx::rsqrt_approx(r2a), irb = ptx::rsqrt_approx(r2b);
    if (SELF) {
      ira = r2a > 0.f ? ira : 0.f;
      irb = r2b > 0.f ? irb : 0.f;
    }
    const uint64_t IR = ptx::f2_pack(ira, irb);
    const uint64_t T = ptx::f2_mul(ptx::f2_mul(R2, IR), KAP);
    const uint64_t N = ptx::f2_sub(ptx::f2_add(T, MAG), MAG);
    const uint64_t TH = ptx::f2_mul(ptx::f2_sub(T, N), TWOPI);
    float ta, tb, sa, ca, sb, cb;
    ptx::f2_unpack(TH, ta, tb);
    __sincosf(ta, &sa, &ca);
    __sincosf(tb, &sb, &cb);
    const uint64_t FR = ptx::f2_mul(IR, ptx::f2_pack(ca, cb));
    const uint64_t FI = ptx::f2_mul(IR, ptx::f2_pack(sa, sb));
    const uint64_t NFI = ptx::f2_mul(IR, ptx::f2_pack(-sa, -sb));
#pragma unroll
    for (int r = 0; r < kP2pRG; ++r) {
      const float4 v = sv4[r][k >> 1];
      const uint64_t VX = ptx::f2_pack(v.x, v.y), VY = ptx::f2_pack(v.z, v.w);
      CR[r] = ptx::f2_fma(FR, VX, ptx::f2_fma(NFI, VY, CR[r]));
      CI[r] = ptx::f2_fma(FR, VY, ptx::f2_fma(FI, VX, CI[r]));
    }
  }
}

__global__ void __launch_bounds__(128) k_p2p_mrhs(const float *tl, int64_t nt, const int32_t *tperm,
                                                  const int32_t *leaf_cell, const int32_t *leaf_begin,
                                                  const int32_t *leaf_end, const float *sl, int64_t ns,
                                                  const int32_t *sperm, const int32_t *s_leaf_of_cell,
                                                  const int32_t *sb, const int32_t *se, int g, float w,
                                                  const int32_t *near_off, int nnear, float kappa, const float2 *x,
                                                  int nrhs, const float2 *ysorted, float2 *y) {
  __shared__ __align__(16) float qx[128], qy[128], qz[128];
  __shared__ __align__(16) float4 sv4[kP2pRG][64];
  const int leaf = blockIdx.x;
  const int cell = leaf_cell[leaf];
  const int cx = cell % g, cy = (cell / g) % g, cz = cell / (g * g);
  const int b = leaf_begin[leaf], e = leaf_end[leaf];
  const float inv4pi = (float)(1.0 / (4.0 * kPi));
  const float kap_rev = (float)((double)kappa / (2.0 * kPi));   // kappa r in revolutions
  const uint64_t KAP = ptx::f2_pack(kap_rev, kap_rev);
  const int t = threadIdx.x;
  // this thread's words of sv4: vx at (t / 2) * 4 + (t & 1), vy two further
  const int wx = (t >> 1) * 4 + (t & 1);
  for (int p0 = b; p0 < e; p0 += blockDim.x) {
    const int p = p0 + t;
    const bool act = p < e;
    const float px = act ? tl[p] : 0.f, py = act ? tl[nt + p] : 0.f, pz = act ? tl[2 * nt + p] : 0.f;
    const uint64_t PX = ptx::f2_pack(px, px), PY = ptx::f2_pack(py, py), PZ = ptx::f2_pack(pz, pz);
    for (int r0 = 0; r0 < nrhs; r0 += kP2pRG) {
      const int rn = min(kP2pRG, nrhs - r0);
      double ar[kP2pRG], ai[kP2pRG];
#pragma unroll
      for (int r = 0; r < kP2pRG; ++r) ar[r] = ai[r] = 0.0;
      for (int i = 0; i < nnear; ++i) {
        const int dx = near_off[3 * i], dy = near_off[3 * i + 1], dz = near_off[3 * i + 2];
        const int sx = cx - dx, sy = cy - dy, sz = cz - dz;
        if (sx < 0 || sy < 0 || sz < 0 || sx >= g || sy >= g || sz >= g) continue;
        const int s = s_leaf_of_cell[sx + g * (sy + g * sz)];
        if (s < 0) continue;
        const bool self = (dx | dy | dz) == 0;
        const float ox = w * dx, oy = w * dy, oz = w * dz;   // m_t - m_s
        for (int q0 = sb[s]; q0 < se[s]; q0 += blockDim.x) {
          const int cnt = min((int)blockDim.x, se[s] - q0);
          __syncthreads();
          if (t < cnt) {
            const int q = q0 + t;
            qx[t] = sl[q] - ox;
            qy[t] = sl[ns + q] - oy;
            qz[t] = sl[2 * ns + q] - oz;
            const int64_t src = sperm[q];
#pragma unroll
            for (int r = 0; r < kP2pRG; ++r) {
              const float2 v = (r < rn) ? x[(int64_t)(r0 + r) * ns + src] : make_float2(0.f, 0.f);
              float *sw = reinterpret_cast<float *>(sv4[r]);
              sw[wx] = v.x * inv4pi;   // x_y / (4 pi)
              sw[wx + 2] = v.y * inv4pi;
            }
          } else if (t == cnt) {   // odd count: a source of value 0
            qx[t] = qy[t] = qz[t] = 0.f;
#pragma unroll
            for (int r = 0; r < kP2pRG; ++r) {
              float *sw = reinterpret_cast<float *>(sv4[r]);
              sw[wx] = sw[wx + 2] = 0.f;
            }
          }
          __syncthreads();
          uint64_t CR[kP2pRG], CI[kP2pRG];
#pragma unroll
          for (int r = 0; r < kP2pRG; ++r) CR[r] = CI[r] = 0ull;
          const int cnt2 = (cnt + 1) & ~1;
          if (self)
            p2p_staged_mrhs<true>(qx, qy, qz, sv4, cnt2, PX, PY, PZ, CR, CI, KAP);
          else
            p2p_staged_mrhs<false>(qx, qy, qz, sv4, cnt2, PX, PY, PZ, CR, CI, KAP);
#pragma unroll
          for (int r = 0; r < kP2pRG; ++r) {
            float r0v, r1v, i0v, i1v;
            ptx::f2_unpack(CR[r], r0v, r1v);
            ptx::f2_unpack(CI[r], i0v, i1v);
            ar[r] += (double)r0v + (double)r1v;
            ai[r] += (double)i0v + (double)i1v;
          }
        }
      }
      if (act) {
#pragma unroll
        for (int r = 0; r < kP2pRG; ++r) {
          if (r < rn) {
            const float2 f = ysorted[(int64_t)(r0 + r) * nt + p];
            y[(int64_t)(r0 + r) * nt + tperm[p]] = make_float2((float)(ar[r] + (double)f.x), (float)(ai[r] + (double)f.y));
          }
        }
      }
    }
  }
}

// Nearfield for small leaves (at most kSmallLeaf points): one warp per
// target leaf, lane i takes nearfield offsets i, i + 32, ... and sums that
// leaf's sources into every target of the leaf; the warp then reduces per
// target.  Keeps all lanes busy when leaves hold a few points.
constexpr int kSmallLeaf = 16;

__global__ void __launch_bounds__(256) k_p2p_small(const float *tl, int64_t nt, const int32_t *tperm,
                                                   const int32_t *leaf_cell, const int32_t *leaf_begin,
                                                   const int32_t *leaf_end, int64_t nleaves, const float *sl,
                                                   int64_t ns, const int32_t *sperm, const int32_t *s_leaf_of_cell,
                                                   const int32_t *sb, const int32_t *se, int g, float w,
                                                   const int32_t *near_off, int nnear, float kappa,
                                                   const float2 *x, const float2 *ysorted, float2 *y) {
  const int64_t leaf = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (leaf >= nleaves) return;
  const int cell = leaf_cell[leaf];
  const int cx = cell % g, cy = (cell / g) % g, cz = cell / (g * g);
  const int b = leaf_begin[leaf];
  const int cnt = min(kSmallLeaf, leaf_end[leaf] - b);
  const float inv4pi = (float)(1.0 / (4.0 * kPi));
  const float kap_rev = (float)((double)kappa / (2.0 * kPi));   // kappa r in revolutions
  float px[kSmallLeaf], py[kSmallLeaf], pz[kSmallLeaf], cr[kSmallLeaf], ci[kSmallLeaf];
#pragma unroll
  for (int u = 0; u < kSmallLeaf; ++u) {
    const bool a = u < cnt;
    px[u] = a ? tl[b + u] : 0.f;
    py[u] = a ? tl[nt + b + u] : 0.f;
    pz[u] = a ? tl[2 * nt + b + u] : 0.f;
    cr[u] = ci[u] = 0.f;
  }
  for (int i = lane; i < nnear; i += 32) {
    const int dx = near_off[3 * i], dy = near_off[3 * i + 1], dz = near_off[3 * i + 2];
    const int sx = cx - dx, sy = cy - dy, sz = cz - dz;
    if (sx < 0 || sy < 0 || sz < 0 || sx >= g || sy >= g || sz >= g) continue;
    const int s = s_leaf_of_cell[sx + g * (sy + g * sz)];
    if (s < 0) continue;
    const float ox = w * dx, oy = w * dy, oz = w * dz;   // m_t - m_s
    for (int q = sb[s]; q < se[s]; ++q) {
      const float qx = sl[q] - ox, qy = sl[ns + q] - oy, qz = sl[2 * ns + q] - oz;
      const float2 x0 = x[sperm[q]];
      const float2 v = make_float2(x0.x * inv4pi, x0.y * inv4pi);   // x_y / (4 pi)
#pragma unroll
      for (int u = 0; u < kSmallLeaf; ++u) {
        if (u >= cnt) break;
        const float d0 = px[u] - qx, d1 = py[u] - qy, d2 = pz[u] - qz;
        const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
        if (r2 == 0.f) continue;   // coincident points (zero diagonal)
        const float ir = rsqrtf(r2);
        float sn, cs;
        exp_i_rev(kap_rev * (r2 * ir), sn, cs);   // exp(i kappa r)
        cr[u] = fmaf(ir, fmaf(cs, v.x, -sn * v.y), cr[u]);
        ci[u] = fmaf(ir, fmaf(cs, v.y, sn * v.x), ci[u]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kSmallLeaf; ++u) {
    for (int o = 16; o > 0; o >>= 1) {
      cr[u] += __shfl_xor_sync(0xffffffffu, cr[u], o);
      ci[u] += __shfl_xor_sync(0xffffffffu, ci[u], o);
    }
  }
  if (lane < cnt) {
    // lane u writes target u (registers indexed by a compile-time loop)
#pragma unroll
    for (int u = 0; u < kSmallLeaf; ++u) {
      if (u == lane) {
        const float2 f = ysorted[b + u];
        y[tperm[b + u]] = make_float2(cr[u] + f.x, ci[u] + f.y);
      }
    }
  }
}

// ------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    DFDM_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (!p || q != cudaDriverEntryPointSuccess)
      throw Error{DFDM_ERR_CUDA, "cuTensorMapEncodeTiled is not available"};
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

void encode(CUtensorMap *m, CUtensorMapDataType dt, int rank, void *ptr, const cuuint64_t *dims,
            const cuuint64_t *strides, const cuuint32_t *box, const cuuint32_t *es, CUtensorMapSwizzle sw) {
  CUresult r = tensor_map_encoder()(m, dt, rank, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error{DFDM_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r)};
}

}  // namespace

// Per-plan state of the tensor-core form.
struct TcState {
  int KP = 0;                            // = NP, padded stacked length
  std::vector<float *> mom32;            // per level FP32 moment grids
  std::vector<double *> loc64;           // per level local grids (FP64 sums)
  std::vector<__half *> mhi, mlo;        // per level split moments
  std::vector<CUtensorMap> map_mhi, map_mlo;
  __half *opk = nullptr;                 // split operator images (see op_pair_row)
  CUtensorMap map_op;                    // 2-D map over opk: rows of 256 FP16 (512 B)
  int4 *meta = nullptr;                  // parallel to the M2L lists (see M2lArgs::meta)
  std::vector<int> op_exp;               // per level operator scale exponent
  float *maxabs = nullptr;               // per level max |moment|
  int *mom_exp = nullptr;                // per level moment exponent
  float *e1 = nullptr;                   // FP32 1-D transfer matrices
  float2 *phase = nullptr;               // FP32 directional diagonals
  float *tl = nullptr, *sl = nullptr;    // leaf-local coordinates
  float2 *ysorted = nullptr;
  int num_sms = 1;
  size_t l2_bytes = 0;
  TcTuning tune;                         // launch shapes set by the tuner (0: the default rule)
};

// CTAs per (tile, alpha) for one M2L level.  Two reasons to split every
// operator list into s contiguous chunks (chunks add into the locals
// atomically):
//  * waves: with one resident CTA per SM a level of `ctas` CTAs runs in
//    ceil(ctas / num_sms) waves, so a level with few tiles (the coarse
//    levels) leaves SMs idle; take the smallest s whose waves per unit of
//    work are within 2 % of the best, keeping >= 16 ops a chunk;
//  * L2: when a parity has at least num_sms CTAs (units: tiles), all
//    resident CTAs work on one (parity, chunk) at a time (grid x is the
//    fastest index), so a chunk whose operators fit in 40 % of L2 is
//    read from HBM about once per chunk instead of once per CTA that falls
//    out of step with the rest.
static int m2l_split(int units, int ops_per_alpha, int num_sms, size_t op_bytes, size_t l2_bytes) {
  const int64_t ctas = (int64_t)units * 8;
  auto cost = [&](int s) { return (double)((ctas * s + num_sms - 1) / num_sms) / s; };
  int s_min = 1;
  if (units >= num_sms && op_bytes > 0) {
    const int c_max = std::max<int>(16, (int)(0.4 * (double)l2_bytes / (double)op_bytes));
    s_min = std::max(1, (ops_per_alpha + c_max - 1) / c_max);
  }
  const int smax = std::max(s_min, std::min(32, ops_per_alpha / 16));
  double best = cost(s_min);
  for (int s = s_min + 1; s <= smax; ++s) best = std::min(best, cost(s));
  for (int s = s_min; s <= smax; ++s)
    if (cost(s) <= best * 1.02) return s;
  return s_min;
}

// CTA pairs of one M2L level: tiles of kPX x kPY x 2 kPZ parent cells.
static int m2l_pairs(const LevelPlan &L) {
  const int gp = L.grid / 2;
  return ((gp + kPX - 1) / kPX) * ((gp + kPY - 1) / kPY) * ((gp + 2 * kPZ - 1) / (2 * kPZ));
}

static int m2l_ops_alpha(const LevelPlan &L) {
  size_t ops_alpha = 0;
  for (int al = 0; al < 8; ++al) ops_alpha = std::max(ops_alpha, L.alpha_ops[al].size());
  return (int)ops_alpha;
}

// The default rule's chunk count of level l (m2l_split above).
static int m2l_nsplit_rule(const Plan &plan, int l) {
  const TcState &T = *plan.tc;
  const LevelPlan &L = plan.levels[l];
  return m2l_split(m2l_pairs(L), m2l_ops_alpha(L), T.num_sms / 2, (size_t)T.KP * T.KP * 4, T.l2_bytes);
}

static TcState &tc_state(Plan &plan) {
  if (!plan.tc) plan.tc = new TcState();
  return *plan.tc;
}

void destroy_tc(Plan &plan) {
  delete plan.tc;
  plan.tc = nullptr;
}

void build_tc(Plan &plan, cudaStream_t st) {
  TcState &T = tc_state(plan);
  const int o = plan.order, n = plan.n, p = plan.depth;
  if (o > 7) throw Error{DFDM_ERR_UNSUPPORTED, "tensor-core form supports orders 2..7"};
  {
    int dev = 0;
    DFDM_CUDA_TRY(cudaGetDevice(&dev));
    DFDM_CUDA_TRY(cudaDeviceGetAttribute(&T.num_sms, cudaDevAttrMultiProcessorCount, dev));
    int l2 = 0;
    DFDM_CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    T.l2_bytes = (size_t)l2;
  }
  const int KP = round_up(2 * n, 64);  // stacked length: N halves and H-drain groups of 16
  if (KP / 2 > 256) throw Error{DFDM_ERR_UNSUPPORTED, "order too large for one MMA N half"};
  T.KP = KP;
  // opt the M2L kernel into its dynamic shared memory once, here, so the
  // apply itself makes no attribute calls (it can be captured in a graph)
  switch (KP) {
    case 64: DFDM_CUDA_TRY(cudaFuncSetAttribute(k_m2l_pair<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, PairSmem<64>::kTotal)); break;
    case 128: DFDM_CUDA_TRY(cudaFuncSetAttribute(k_m2l_pair<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, PairSmem<128>::kTotal)); break;
    case 256: DFDM_CUDA_TRY(cudaFuncSetAttribute(k_m2l_pair<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, PairSmem<256>::kTotal)); break;
    case 448: DFDM_CUDA_TRY(cudaFuncSetAttribute(k_m2l_pair<448>, cudaFuncAttributeMaxDynamicSharedMemorySize, PairSmem<448>::kTotal)); break;
    default: break;
  }
  // FP32 constants
  {
    double cheb[kMaxOrder] = {0}, lagw[kMaxOrder] = {0};
    chebyshev_tables(o, cheb, lagw);
    DFDM_CUDA_TRY(cudaMemcpyToSymbol(c_cheb, cheb, sizeof(cheb)));
    DFDM_CUDA_TRY(cudaMemcpyToSymbol(c_lagw, lagw, sizeof(lagw)));
    std::vector<double> e1d(2 * o * o);
    DFDM_CUDA_TRY(cudaMemcpy(e1d.data(), plan.e1, e1d.size() * 8, cudaMemcpyDeviceToHost));
    std::vector<float> e1f(e1d.begin(), e1d.end());
    T.e1 = plan.alloc<float>(e1f.size());
    DFDM_CUDA_TRY(cudaMemcpy(T.e1, e1f.data(), e1f.size() * 4, cudaMemcpyHostToDevice));
  }
  // directional diagonals in FP32 (FP64 arguments)
  if (plan.m2m_phase) {
    int64_t total = 0;
    for (int l = 0; l < p; ++l)
      if (plan.m2m_phase_off[l] >= 0) total = std::max<int64_t>(total, plan.m2m_phase_off[l] + 8ll * plan.levels[l].slot_dir.size() * n);
    T.phase = plan.alloc<float2>(total);
    for (int l = plan.min_level; l < p; ++l) {
      if (plan.m2m_phase_off[l] < 0) continue;
      const LevelPlan &L = plan.levels[l];
      const LevelPlan &C = plan.levels[l + 1];
      const int ns = (int)L.slot_dir.size();
      std::vector<double> c2(3 * ns);
      for (int s = 0; s < ns; ++s)
        for (int i = 0; i < 3; ++i) c2[3 * s + i] = C.dir_vec[3 * L.child_slot[s] + i];
      double *d_c = nullptr, *d_c2 = nullptr;
      DFDM_CUDA_TRY(cudaMalloc(&d_c, 3 * ns * 8));
      DFDM_CUDA_TRY(cudaMalloc(&d_c2, 3 * ns * 8));
      DFDM_CUDA_TRY(cudaMemcpy(d_c, L.dir_vec.data(), 3 * ns * 8, cudaMemcpyHostToDevice));
      DFDM_CUDA_TRY(cudaMemcpy(d_c2, c2.data(), 3 * ns * 8, cudaMemcpyHostToDevice));
      k_phase_table_f<<<dim3(ns, 8), 128, 0, st>>>(o, n, ns, d_c, d_c2, plan.kappa, 0.25 * L.w,
                                                   T.phase + plan.m2m_phase_off[l]);
      DFDM_LAUNCH_CHECK();
      DFDM_CUDA_TRY(cudaStreamSynchronize(st));
      cudaFree(d_c);
      cudaFree(d_c2);
    }
  }
  // leaf-local coordinates
  T.tl = plan.alloc<float>(3 * plan.tt.n);
  T.sl = plan.alloc<float>(3 * plan.ts.n);
  const double wl = plan.levels[p].w;
  k_local_coords<<<nblk(plan.tt.nleaves, 128), 128, 0, st>>>(plan.tt.xyz, plan.tt.n, plan.tt.leaf_cell,
                                                             plan.tt.leaf_begin, plan.tt.leaf_end, plan.tt.nleaves,
                                                             plan.root_lo[0], plan.root_lo[1], plan.root_lo[2], wl,
                                                             1 << p, T.tl);
  DFDM_LAUNCH_CHECK();
  k_local_coords<<<nblk(plan.ts.nleaves, 128), 128, 0, st>>>(plan.ts.xyz, plan.ts.n, plan.ts.leaf_cell,
                                                             plan.ts.leaf_begin, plan.ts.leaf_end, plan.ts.nleaves,
                                                             plan.root_lo[0], plan.root_lo[1], plan.root_lo[2], wl,
                                                             1 << p, T.sl);
  DFDM_LAUNCH_CHECK();
  T.ysorted = plan.alloc<float2>((size_t)plan.tt.n * plan.params.nrhs_max);   // far field per right-hand side
  // grids
  T.mom32.assign(p + 1, nullptr);
  T.loc64.assign(p + 1, nullptr);
  T.mhi.assign(p + 1, nullptr);
  T.mlo.assign(p + 1, nullptr);
  T.map_mhi.resize(p + 1);
  T.map_mlo.resize(p + 1);
  T.op_exp.assign(p + 1, 0);
  T.maxabs = plan.alloc<float>(p + 1);
  T.mom_exp = plan.alloc<int>(p + 1);
  DFDM_CUDA_TRY(cudaMemset(T.mom_exp, 0, (p + 1) * sizeof(int)));
  for (int l = plan.min_level; l <= p; ++l) {
    const size_t cnt = plan.levels[l].slot_dir.size() * ((size_t)1 << (3 * l)) * KP;
    T.mom32[l] = plan.alloc<float>(cnt);
    T.loc64[l] = plan.alloc<double>(cnt);
    if (!plan.levels[l].off.empty()) {
      T.mhi[l] = plan.alloc<__half>(cnt);
      T.mlo[l] = plan.alloc<__half>(cnt);
      const cuuint64_t hg = (cuuint64_t)1 << (l - 1);   // half the level grid
      const cuuint64_t dims[5] = {(cuuint64_t)kK, hg, hg, hg,
                                  (cuuint64_t)plan.levels[l].slot_dir.size() * (KP / kK) * 8};
      const cuuint64_t strides[4] = {(cuuint64_t)kK * 2, (cuuint64_t)kK * 2 * hg, (cuuint64_t)kK * 2 * hg * hg,
                                     (cuuint64_t)kK * 2 * hg * hg * hg};
      const cuuint32_t box[5] = {(cuuint32_t)kK, kPX, kPY, kPZ, 1};
      const cuuint32_t es[5] = {1, 1, 1, 1, 1};
      encode(&T.map_mhi[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 5, T.mhi[l], dims, strides, box, es,
             CU_TENSOR_MAP_SWIZZLE_64B);
      encode(&T.map_mlo[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 5, T.mlo[l], dims, strides, box, es,
             CU_TENSOR_MAP_SWIZZLE_64B);
    }
  }
  // split operators, one scale per level: |A~| <= 1 / (4 pi w (2 - r_max))
  const int nops = plan.n_ops;
  if (nops > 0) {
    std::vector<int32_t> op_level;
    std::vector<double> op_dir, level_w;
    std::vector<float> level_scale(p + 1, 1.0f);
    const double rmax = std::cos(kPi / (2.0 * o));
    for (auto &L : plan.levels) {
      level_w.push_back(L.w);
      const double amax = 1.0 / (4.0 * kPi * L.w * (2.0 - rmax));
      const int e = 14 - (int)std::ceil(std::log2(amax));
      T.op_exp[L.level] = e;
      level_scale[L.level] = std::ldexp(1.0f, e);
      for (size_t i = 0; i < L.op_dir.size(); ++i) {
        op_level.push_back(L.level);
        double c[3];
        direction_vector(plan.l_hf, L.level, L.op_dir[i], c);
        op_dir.insert(op_dir.end(), c, c + 3);
      }
    }
    int32_t *d_level = nullptr;
    double *d_dir = nullptr, *d_w = nullptr;
    float *d_sc = nullptr;
    DFDM_CUDA_TRY(cudaMalloc(&d_level, nops * 4));
    DFDM_CUDA_TRY(cudaMalloc(&d_dir, nops * 3 * 8));
    DFDM_CUDA_TRY(cudaMalloc(&d_w, level_w.size() * 8));
    DFDM_CUDA_TRY(cudaMalloc(&d_sc, level_scale.size() * 4));
    DFDM_CUDA_TRY(cudaMemcpy(d_level, op_level.data(), nops * 4, cudaMemcpyHostToDevice));
    DFDM_CUDA_TRY(cudaMemcpy(d_dir, op_dir.data(), nops * 3 * 8, cudaMemcpyHostToDevice));
    DFDM_CUDA_TRY(cudaMemcpy(d_w, level_w.data(), level_w.size() * 8, cudaMemcpyHostToDevice));
    DFDM_CUDA_TRY(cudaMemcpy(d_sc, level_scale.data(), level_scale.size() * 4, cudaMemcpyHostToDevice));
    const size_t ocnt = (size_t)nops * KP * KP * 2;
    T.opk = plan.alloc<__half>(ocnt);
    k_coupling_split_pair<<<dim3(nops, KP), 128, 0, st>>>(o, n, KP, KP / 2, d_level, plan.op_off_dev, d_dir, d_w,
                                                           d_sc, plan.kappa, T.opk);
    DFDM_LAUNCH_CHECK();
    DFDM_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(d_level);
    cudaFree(d_dir);
    cudaFree(d_w);
    cudaFree(d_sc);
    const int NB = KP / 4;
    const cuuint64_t dims[2] = {256, (cuuint64_t)nops * (cuuint64_t)(KP * KP * 2 / 256)};
    const cuuint64_t strides[1] = {512};
    const cuuint32_t box[2] = {256, (cuuint32_t)(2 * NB * 32 / 256)};
    const cuuint32_t es[2] = {1, 1};
    encode(&T.map_op, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, T.opk, dims, strides, box, es, CU_TENSOR_MAP_SWIZZLE_NONE);
  }
  // per entry of the M2L lists (same order as plan.m2l_ops): the global
  // operator index, its offset packed as three biased bytes, its direction
  // slot and the end of the run of entries sharing that slot (the lists are
  // sorted by slot), relative to the level's first entry
  {
    std::vector<int4> meta;
    for (auto &L : plan.levels) {
      const size_t base = meta.size();
      for (int al = 0; al < 8; ++al) {
        const auto &lst = L.alpha_ops[al];
        const size_t s0 = meta.size();
        meta.resize(s0 + lst.size());
        for (size_t i = lst.size(); i-- > 0;) {
          const int op = lst[i];
          int packed = 0;
          for (int a = 0; a < 3; ++a) {
            const int d = L.off[3 * op + a];
            if (d < -128 || d > 127) throw Error{DFDM_ERR_UNSUPPORTED, "M2L offset out of the packed range"};
            packed |= (d + 128) << (8 * a);
          }
          const bool same = i + 1 < lst.size() && L.op_slot[lst[i + 1]] == L.op_slot[op];
          meta[s0 + i] = make_int4(L.op_base + op, packed, L.op_slot[op],
                                   same ? meta[s0 + i + 1].w : (int32_t)(s0 + i + 1 - base));
        }
      }
    }
    T.meta = plan.alloc<int4>(std::max<size_t>(meta.size(), 1));
    if (!meta.empty()) DFDM_CUDA_TRY(cudaMemcpy(T.meta, meta.data(), meta.size() * sizeof(int4), cudaMemcpyHostToDevice));
  }
  DFDM_CUDA_TRY(cudaStreamSynchronize(st));
}

// One right-hand side: far field into ys (sorted target order), then, when
// `near` is set, the nearfield and the output y in the caller's order.
// Default block shape of k_p2p_f32 (threads, target chunks per leaf).
static void p2p_shape_rule(const Plan &plan, unsigned &threads, unsigned &chunks) {
  const Tree &tt = plan.tt;
  threads = (tt.n <= 64 * tt.nleaves) ? 32u : 128u;
  const int64_t per128 = (tt.max_leaf_size + kP2pT * 128 - 1) / (kP2pT * 128);
  if (threads == 128u && tt.nleaves * per128 * 4 < 16ll * plan.tc->num_sms) threads = 32u;
  chunks = (unsigned)std::min<int64_t>(
      16, std::max<int64_t>(1, (tt.max_leaf_size + kP2pT * threads - 1) / (kP2pT * threads)));
}

template <int O, int NP>
static void apply_tc_o(Plan &plan, const float2 *x, float2 *y, float2 *ys, bool near, cudaStream_t st) {
  constexpr int N = O * O * O;
  TcState &T = *plan.tc;
  Timing &tm = plan.timing;
  const int p = plan.depth, KP = T.KP;
  const Tree &tt = plan.tt, &ts = plan.ts;
  const bool far = plan.min_level <= p;
  if (far) {
    const LevelPlan &P = plan.levels[p];
    const int nsl = (int)P.slot_dir.size();
    {
      PhaseScope sc(tm, kPhS2M, st);
      DFDM_CUDA_TRY(cudaMemsetAsync(T.maxabs, 0, (p + 1) * sizeof(float), st));
      for (int l = plan.min_level; l <= p; ++l) {
        const size_t bytes = plan.levels[l].slot_dir.size() * ((size_t)1 << (3 * l)) * KP * sizeof(double);
        DFDM_CUDA_TRY(cudaMemsetAsync(T.loc64[l], 0, bytes, st));
      }
      const size_t bytes = P.slot_dir.size() * ((size_t)1 << (3 * p)) * KP * sizeof(float);
      DFDM_CUDA_TRY(cudaMemsetAsync(T.mom32[p], 0, bytes, st));
      if (nsl > 0 && ts.nleaves > 0) {
        if (ts.max_leaf_size <= kSmallLeafS2M)
          k_s2m_small<O><<<nblk(ts.nleaves * nsl * 32, 256), 256, 0, st>>>(
              ts.xyz, ts.n, ts.perm, x, ts.leaf_cell, ts.leaf_begin, ts.leaf_end, ts.nleaves, nsl,
              plan.root_lo[0], plan.root_lo[1], plan.root_lo[2], P.w, P.grid, plan.dir_vec_dev + plan.dir_vec_off[p],
              plan.kappa, T.mom32[p], 1ll << (3 * p), KP, T.maxabs + p);
        else
        k_s2m_tc<O><<<dim3((unsigned)ts.nleaves, nsl), 128, 0, st>>>(
            ts.xyz, ts.n, ts.perm, x, ts.leaf_cell, ts.leaf_begin, ts.leaf_end, plan.root_lo[0], plan.root_lo[1],
            plan.root_lo[2], P.w, P.grid, plan.dir_vec_dev + plan.dir_vec_off[p], plan.kappa, T.mom32[p],
            1ll << (3 * p), KP, T.maxabs + p);
        DFDM_COUNT_LAUNCH(plan);
      }
    }
    {
      PhaseScope sc(tm, kPhM2M, st);
      for (int l = p - 1; l >= plan.min_level; --l) {
        const LevelPlan &L = plan.levels[l];
        const int ns = (int)L.slot_dir.size();
        if (ns == 0) continue;
        const float2 *ph = plan.m2m_phase_off[l] >= 0 ? T.phase + plan.m2m_phase_off[l] : nullptr;
        k_m2m_f32<O><<<dim3((unsigned)(1ll << (3 * l)), ns), 128, 0, st>>>(
            T.mom32[l + 1], T.mom32[l], L.grid, plan.child_slot_dev + plan.child_slot_off[l], ph, ns, T.e1, KP,
            T.maxabs + l);
        DFDM_COUNT_LAUNCH(plan);
      }
    }
    // split + M2L
    for (int l = std::max(1, plan.min_level); l <= p; ++l) {
      const LevelPlan &L = plan.levels[l];
      if (L.off.empty()) continue;
      {
        PhaseScope sc(tm, kPhSplit, st);
        const int64_t cnt = (int64_t)L.slot_dir.size() * (1ll << (3 * l)) * KP;
        k_split<<<1184, 256, 0, st>>>(T.mom32[l], cnt, L.grid, KP, T.maxabs + l, T.mom_exp + l, T.mhi[l], T.mlo[l],
                                      plan.err_flag);
        DFDM_COUNT_LAUNCH(plan);
      }
      M2lArgs a;
      a.alpha_ops = plan.m2l_ops + plan.m2l_ops_off[l * 9];
      a.alpha_off = plan.m2l_aoff_dev + 9 * l;
      a.op_off = plan.op_off_dev;
      a.op_slot = plan.op_slot_dev;
      a.meta = T.meta + plan.m2l_ops_off[l * 9];
      a.loc = T.loc64[l];
      a.g = L.grid;
      a.n = N;
      a.KP = KP;
      a.mom_exp = T.mom_exp + l;
      a.op_exp = T.op_exp[l];
      a.err = plan.err_flag;
      const int pairs = m2l_pairs(L);
      a.nsplit = (l < (int)T.tune.m2l_nsplit.size() && T.tune.m2l_nsplit[l] > 0) ? T.tune.m2l_nsplit[l]
                                                                                 : m2l_nsplit_rule(plan, l);
      const int smem = PairSmem<NP>::kTotal;
      PhaseScope sc(tm, kPhM2L0 + l, st);
      k_m2l_pair<NP><<<dim3(2 * pairs, 8, a.nsplit), kPThreads, smem, st>>>(T.map_mhi[l], T.map_mlo[l], T.map_op, a);
      DFDM_COUNT_LAUNCH(plan);
    }
    {
      PhaseScope sc(tm, kPhL2L, st);
      for (int l = plan.min_level; l < p; ++l) {
        const LevelPlan &L = plan.levels[l];
        const LevelPlan &C = plan.levels[l + 1];
        const int nsp = (int)L.slot_dir.size(), nsc = (int)C.slot_dir.size();
        if (nsp == 0 || nsc == 0) continue;
        const float2 *ph = plan.m2m_phase_off[l] >= 0 ? T.phase + plan.m2m_phase_off[l] : nullptr;
        k_l2l_f32<O><<<dim3((unsigned)(1ll << (3 * (l + 1))), nsc), 128, 0, st>>>(
            T.loc64[l], T.loc64[l + 1], C.grid, plan.l2l_pslots_dev + plan.l2l_pslots_off[l],
            plan.l2l_poff_dev + plan.l2l_poff_off[l], ph, nsp, T.e1, KP);
        DFDM_COUNT_LAUNCH(plan);
      }
    }
    PhaseScope sc(tm, kPhL2T, st);
    if (nsl > 0 && tt.nleaves > 0 && tt.max_leaf_size <= kSmallLeaf) {
      k_l2t_small<O><<<nblk(tt.nleaves * 32, 256), 256, 0, st>>>(
          tt.xyz, tt.n, tt.leaf_cell, tt.leaf_begin, tt.leaf_end, tt.nleaves, plan.root_lo[0], plan.root_lo[1],
          plan.root_lo[2], P.w, P.grid, plan.dir_vec_dev + plan.dir_vec_off[p], nsl, plan.kappa, T.loc64[p],
          1ll << (3 * p), KP, ys);
      DFDM_COUNT_LAUNCH(plan);
    } else if (nsl > 0 && tt.nleaves > 0) {
      k_l2t_tc<O><<<(unsigned)tt.nleaves, 128, 0, st>>>(tt.xyz, tt.n, tt.leaf_cell, tt.leaf_begin, tt.leaf_end,
                                                        plan.root_lo[0], plan.root_lo[1], plan.root_lo[2], P.w,
                                                        P.grid, plan.dir_vec_dev + plan.dir_vec_off[p], nsl,
                                                        plan.kappa, T.loc64[p], 1ll << (3 * p), KP, ys);
      DFDM_COUNT_LAUNCH(plan);
    } else {
      DFDM_CUDA_TRY(cudaMemsetAsync(ys, 0, tt.n * sizeof(float2), st));
    }
  } else {
    DFDM_CUDA_TRY(cudaMemsetAsync(ys, 0, tt.n * sizeof(float2), st));
  }
  if (!near) return;
  PhaseScope sc(tm, kPhNear, st);
  if (tt.max_leaf_size <= kSmallLeaf) {
    k_p2p_small<<<(unsigned)((tt.nleaves * 32 + 255) / 256), 256, 0, st>>>(
        T.tl, tt.n, tt.perm, tt.leaf_cell, tt.leaf_begin, tt.leaf_end, tt.nleaves, T.sl, ts.n, ts.perm,
        ts.leaf_of_cell, ts.leaf_begin, ts.leaf_end, 1 << p, (float)plan.levels[p].w, plan.near_off_dev,
        (int)(plan.near_off.size() / 3), (float)plan.kappa, x, ys, y);
  } else {
    // blocks (target leaf, target chunk): leaves of a few dozen points
    // (uniform trees just above the warp-per-leaf size) get one warp; large
    // leaves 4 warps, or one warp per chunk of kP2pT x 32 targets when one
    // block per leaf would not give every SM about 16 warps
    unsigned p2p_threads, chunks;
    p2p_shape_rule(plan, p2p_threads, chunks);
    if (T.tune.p2p_threads > 0) {
      p2p_threads = (unsigned)T.tune.p2p_threads;
      chunks = (unsigned)T.tune.p2p_chunks;
    }
    k_p2p_f32<<<dim3((unsigned)tt.nleaves, chunks), p2p_threads, 0, st>>>(T.tl, tt.n, tt.perm, tt.leaf_cell, tt.leaf_begin, tt.leaf_end,
                                                    T.sl, ts.n, ts.perm, ts.leaf_of_cell, ts.leaf_begin,
                                                    ts.leaf_end, 1 << p, (float)plan.levels[p].w, plan.near_off_dev,
                                                    (int)(plan.near_off.size() / 3), (float)plan.kappa, x,
                                                    ys, y);
  }
  DFDM_COUNT_LAUNCH(plan);
}

std::vector<int> tc_nsplit_candidates(const Plan &plan, int l) {
  std::vector<int> c;
  const LevelPlan &L = plan.levels[l];
  if (l < std::max(1, plan.min_level) || l > plan.depth || L.off.empty()) return c;
  const int rule = m2l_nsplit_rule(plan, l);
  // at least one operator per chunk of every non-empty parity class
  size_t ops_min = SIZE_MAX;
  for (int al = 0; al < 8; ++al)
    if (!L.alpha_ops[al].empty()) ops_min = std::min(ops_min, L.alpha_ops[al].size());
  const int smax = std::max(rule, (int)std::min<size_t>(32, ops_min));
  for (int s : {rule, rule / 2, rule * 2, rule - 1, rule + 1, 1, 4 * rule})
    if (s >= 1 && s <= smax && std::find(c.begin(), c.end(), s) == c.end()) c.push_back(s);
  return c;
}

std::vector<std::pair<int, int>> tc_p2p_candidates(const Plan &plan) {
  std::vector<std::pair<int, int>> c;
  const Tree &tt = plan.tt;
  if (tt.nleaves == 0 || tt.max_leaf_size <= kSmallLeaf) return c;
  unsigned t0, c0;
  p2p_shape_rule(plan, t0, c0);
  c.emplace_back((int)t0, (int)c0);
  for (int t : {32, 64, 128})
    for (int f : {1, 2}) {
      const int ch = (int)std::min<int64_t>(16, f * std::max<int64_t>(1, (tt.max_leaf_size + kP2pT * t - 1) /
                                                                             (kP2pT * t)));
      if (std::find(c.begin(), c.end(), std::make_pair(t, ch)) == c.end()) c.emplace_back(t, ch);
    }
  return c;
}

TcTuning &tc_tuning(Plan &plan) { return plan.tc->tune; }

std::string tc_shape_key(const Plan &plan) {
  const TcState &T = *plan.tc;
  int dev = 0;
  cudaDeviceProp prop;
  DFDM_CUDA_TRY(cudaGetDevice(&dev));
  DFDM_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  std::string k = std::string(prop.name) + "/sm" + std::to_string(T.num_sms) + "/o" + std::to_string(plan.order) +
                  "/d" + std::to_string(plan.depth);
  for (int l = std::max(1, plan.min_level); l <= plan.depth; ++l) {
    const LevelPlan &L = plan.levels[l];
    if (L.off.empty()) continue;
    k += "/L" + std::to_string(l) + ":" + std::to_string(L.grid) + "," + std::to_string(L.slot_dir.size()) + "," +
         std::to_string(m2l_ops_alpha(L));
  }
  k += "/leaf" + std::to_string(plan.tt.nleaves) + "," + std::to_string(plan.tt.max_leaf_size) + "," +
       std::to_string(plan.tt.n);
  for (char &ch : k)
    if (ch == '"' || ch == '\\') ch = '_';
  return k;
}

void apply_tc(Plan &plan, const float2 *x, float2 *y, int nrhs, cudaStream_t st) {
  TcState &T = *plan.tc;
  const Tree &tt = plan.tt, &ts = plan.ts;
  // several right-hand sides on leaves above the warp-per-leaf size: far
  // fields one after the other, then one nearfield pass for all of them
  const bool joint_near = nrhs > 1 && tt.max_leaf_size > kSmallLeaf;
  for (int r = 0; r < nrhs; ++r) {
    const float2 *xr = x + (int64_t)r * ts.n;
    float2 *yr = y + (int64_t)r * tt.n;
    float2 *ys = T.ysorted + (int64_t)r * tt.n;
    switch (plan.order) {
      case 2: apply_tc_o<2, 64>(plan, xr, yr, ys, !joint_near, st); break;     // 2n = 16  -> KP 64
      case 3: apply_tc_o<3, 64>(plan, xr, yr, ys, !joint_near, st); break;     // 2n = 54  -> KP 64
      case 4: apply_tc_o<4, 128>(plan, xr, yr, ys, !joint_near, st); break;    // 2n = 128 -> KP 128
      case 5: apply_tc_o<5, 256>(plan, xr, yr, ys, !joint_near, st); break;    // 2n = 250 -> KP 256
      case 6: apply_tc_o<6, 448>(plan, xr, yr, ys, !joint_near, st); break;    // 2n = 432 -> KP 448
      default: throw Error{DFDM_ERR_UNSUPPORTED, "tensor-core form supports orders 2..6"};
    }
  }
  if (joint_near) {
    const int p = plan.depth;
    PhaseScope sc(plan.timing, kPhNear, st);
    const unsigned threads = (tt.n <= 64 * tt.nleaves) ? 64u : 128u;
    k_p2p_mrhs<<<(unsigned)tt.nleaves, threads, 0, st>>>(
        T.tl, tt.n, tt.perm, tt.leaf_cell, tt.leaf_begin, tt.leaf_end, T.sl, ts.n, ts.perm, ts.leaf_of_cell,
        ts.leaf_begin, ts.leaf_end, 1 << p, (float)plan.levels[p].w, plan.near_off_dev,
        (int)(plan.near_off.size() / 3), (float)plan.kappa, x, nrhs, T.ysorted, y);
    DFDM_COUNT_LAUNCH(plan);
  }
}

}  // namespace dfdm
