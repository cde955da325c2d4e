// FP64 form of Alg. 4 on the CUDA cores, and the operator tables every form
// shares (Sect. 2.7).
//
// Phases are written in the box-centred form: moments and local coefficients
// carry the plane wave relative to their box midpoint,
//   v~c_{s,c} = exp(i kappa <m_s, c>) v~_{s,c},  g~c_{t,c} = exp(i kappa <m_t, c>) g~_{t,c},
// which is algebraically identical to Eqs. (6), (9), (13) and keeps every
// phase argument below kappa * diam(box) instead of kappa * |x|:
//   S2M  v~c[k]  = sum_j L_k(y_j) exp(-i kappa <y_j - m_s, c>) v_j
//   M2M  v~c_s   = sum_{s'} E_oct^T conj(P_oct,c) v~c_{s',c'}
//   M2L  g~c_t  += A~_d v~c_{t-d},
//        A~_d[j,k] = exp(i kappa (|v| - (w/2) <r_j - r_k, c>)) / (4 pi |v|),
//        v = w d + (w/2) (r_j - r_k)     (the coupling matrix of Eq. (9)
//        times exp(i kappa <m_t - m_s, c>): a function of (level, d) only)
//   L2L  g~c_{t'} += P_oct,c (E_oct g~c_t)
//   L2T  g_j    += sum_k L_k(x_j) exp(i kappa <x_j - m_t, c>) g~c_t[k]
// with E_oct the non-directional transfer matrix of the child octant and
// P_oct,c[k] = exp(i kappa h (<(2b - 1) + r_k, c> - <r_k, c'>)) the
// directional diagonal E^d in centred form (h = child half side).  E_oct is a
// tensor product of two 1-D matrices per axis, applied axis by axis.
//
// Moments and locals live on dense level grids, [slot][cell][n] with
// cell = x + G y + G^2 z; empty boxes hold zeros, so every source of an
// admissible offset can be read without an existence test.
#include <cmath>

#include "dfdm_internal.cuh"

namespace dfdm {

namespace {

__constant__ double c_cheb[kMaxOrder];     // reference nodes r_nu
__constant__ double c_lagw[kMaxOrder];     // 1 / prod_{mu != nu} (r_nu - r_mu)

constexpr double kPi = 3.14159265358979323846;

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

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

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // a * conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 cexpi(double a) {
  double s, c;
  sincos(a, &s, &c);
  return make_double2(c, s);
}

// ------------------------------------------------------------ operators
// Coupling operators A~_{l,d} (see the file comment), one block row per (op, j).
__global__ void k_coupling_fp64(int order, int n, const int32_t *op_level,
                                const int32_t *op_off, const double *op_dir,
                                const double *level_w, double kappa,
                                double2 *ops) {
  const int op = blockIdx.x;   // x: up to 2^31 - 1 operators
  const int j = blockIdx.y;
  const int l = op_level[op];
  const double w = level_w[l];
  const double h = 0.5 * w;
  const double d0 = op_off[3 * op], d1 = op_off[3 * op + 1], d2 = op_off[3 * op + 2];
  const double c0 = op_dir[3 * op], c1 = op_dir[3 * op + 1], c2 = op_dir[3 * op + 2];
  const int jx = j % order, jy = (j / order) % order, jz = j / (order * order);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int kx = k % order, ky = (k / order) % order, kz = k / (order * order);
    const double e0 = h * (c_cheb[jx] - c_cheb[kx]);
    const double e1 = h * (c_cheb[jy] - c_cheb[ky]);
    const double e2 = h * (c_cheb[jz] - c_cheb[kz]);
    const double v0 = w * d0 + e0, v1 = w * d1 + e1, v2 = w * d2 + e2;
    const double r = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
    const double arg = kappa * (r - (e0 * c0 + e1 * c1 + e2 * c2));
    const double2 ph = cexpi(arg);
    const double s = 1.0 / (4.0 * kPi * r);
    ops[((int64_t)op * n + j) * n + k] = make_double2(ph.x * s, ph.y * s);
  }
}

// Centred directional diagonals P_{oct,c}[k] for a high-frequency parent level.
__global__ void k_phase_table(int order, int n, int nslots, const double *cvec,
                              const double *c2vec, double kappa, double h,
                              double2 *tab) {
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
    tab[((int64_t)oct * nslots + slot) * n + k] = cexpi(kappa * h * a);
  }
}

// ------------------------------------------------------------ counters
__global__ void k_exist_leaf(const int32_t *leaf_of_cell, int64_t ncell, uint8_t *ex) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncell) ex[c] = leaf_of_cell[c] >= 0 ? 1 : 0;
}

__global__ void k_exist_up(const uint8_t *child, int gp, uint8_t *par) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ncell = (int64_t)gp * gp * gp;
  if (c >= ncell) return;
  const int x = c % gp, y = (c / gp) % gp, z = c / ((int64_t)gp * gp);
  const int g = 2 * gp;
  uint8_t any = 0;
  for (int o = 0; o < 8; ++o) {
    const int64_t cc = (2 * x + (o & 1)) + (int64_t)g * ((2 * y + ((o >> 1) & 1)) + (int64_t)g * (2 * z + (o >> 2)));
    any |= child[cc];
  }
  par[c] = any;
}

__global__ void k_count_level(const uint8_t *ext, const uint8_t *exs, int g,
                              const int32_t *alpha_ops, const int32_t *alpha_off,
                              const int32_t *off, unsigned long long *count) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ncell = (int64_t)g * g * g;
  unsigned long long cnt = 0;
  if (c < ncell && ext[c]) {
    const int x = c % g, y = (c / g) % g, z = c / ((int64_t)g * g);
    const int alpha = (x & 1) + 2 * (y & 1) + 4 * (z & 1);
    for (int i = alpha_off[alpha]; i < alpha_off[alpha + 1]; ++i) {
      const int op = alpha_ops[i];
      const int sx = x - off[3 * op], sy = y - off[3 * op + 1], sz = z - off[3 * op + 2];
      if (sx < 0 || sy < 0 || sz < 0 || sx >= g || sy >= g || sz >= g) continue;
      cnt += exs[sx + (int64_t)g * (sy + (int64_t)g * sz)];
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(count, cnt);
}

__global__ void k_count_near(const int32_t *leaf_cell, const int32_t *tb, const int32_t *te,
                             int64_t nleaves, const int32_t *src_leaf_of_cell,
                             const int32_t *sb, const int32_t *se, int g,
                             const int32_t *near_off, int nnear,
                             unsigned long long *out /*[2]: blocks, entries*/) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long blocks = 0, entries = 0;
  if (t < nleaves) {
    const int c = leaf_cell[t];
    const int x = c % g, y = (c / g) % g, z = c / (g * g);
    const long long nt = te[t] - tb[t];
    for (int i = 0; i < nnear; ++i) {
      const int sx = x - near_off[3 * i], sy = y - near_off[3 * i + 1], sz = z - near_off[3 * i + 2];
      if (sx < 0 || sy < 0 || sz < 0 || sx >= g || sy >= g || sz >= g) continue;
      const int s = src_leaf_of_cell[sx + g * (sy + g * sz)];
      if (s < 0) continue;
      blocks += 1;
      entries += (unsigned long long)nt * (unsigned long long)(se[s] - sb[s]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    blocks += __shfl_down_sync(0xffffffffu, blocks, o);
    entries += __shfl_down_sync(0xffffffffu, entries, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (blocks) atomicAdd(out, blocks);
    if (entries) atomicAdd(out + 1, entries);
  }
}

// ------------------------------------------------------------- S2M (FP64)
template <int O>
__global__ void __launch_bounds__(128) k_s2m_fp64(
    const double *xyz, int64_t n_pts, const int32_t *perm, const double2 *x,
    const int32_t *leaf_cell, const int32_t *leaf_begin, const int32_t *leaf_end,
    double lo0, double lo1, double lo2, double w, int g, const double *dir,
    double kappa, double2 *mom, int64_t ncell) {
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
      const double2 ph = cexpi(-kappa * (y0 * c0 + y1 * c1 + y2 * c2));
      sq[threadIdx.x] = cmul(ph, x[perm[p]]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int k = threadIdx.x + 128 * i;
      if (k < N) {
        const int kx = k % O, ky = (k / O) % O, kz = k / (O * O);
        for (int q = 0; q < cnt; ++q) {
          const double l = sl[0][q][kx] * sl[1][q][ky] * sl[2][q][kz];
          acc[i].x += l * sq[q].x;
          acc[i].y += l * sq[q].y;
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int k = threadIdx.x + 128 * i;
    if (k < N) mom[((int64_t)slot * ncell + cell) * N + k] = acc[i];
  }
}

// ----------------------------------------------------- M2M / L2L (FP64)
// Apply E_oct^T (transpose=true, M2M) or E_oct (L2L) to a smem vector u of
// N = O^3 entries, axis by axis.  e1[b][k][l] = L_l(rho_b(r_k)).
template <int O>
__device__ void tensor_transfer(const double *e1, int oct, bool transpose,
                                double2 *u, double2 *t) {
  constexpr int N = O * O * O;
  const int b[3] = {oct & 1, (oct >> 1) & 1, (oct >> 2) & 1};
  // axis 0 (x, stride 1), then y (stride O), then z (stride O^2)
  for (int a = 0; a < 3; ++a) {
    const int stride = (a == 0) ? 1 : (a == 1 ? O : O * O);
    const double *m = e1 + b[a] * O * O;
    for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
      const int i = (idx / stride) % O;           // output index along the axis
      const int base = idx - i * stride;
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int q = 0; q < O; ++q) {
        // transpose: out[l] = sum_k E[k][l] in[k]; else out[k] = sum_l E[k][l] in[l]
        const double e = transpose ? m[q * O + i] : m[i * O + q];
        const double2 v = u[base + q * stride];
        s.x += e * v.x;
        s.y += e * v.y;
      }
      t[idx] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < N; idx += blockDim.x) u[idx] = t[idx];
    __syncthreads();
  }
}

template <int O>
__global__ void __launch_bounds__(128) k_m2m_fp64(
    const double2 *cmom, double2 *pmom, int gp, const int32_t *child_slot,
    int nslot_c, const double2 *phase, int nslot_p, const double *e1) {
  constexpr int N = O * O * O;
  __shared__ double2 u[N], t[N];
  __shared__ double se1[2 * O * O];
  const int64_t cellp = blockIdx.x;
  const int slot = blockIdx.y;
  const int cs = child_slot[slot];
  const int64_t gc = 2 * (int64_t)gp;
  const int64_t ncp = (int64_t)gp * gp * gp, ncc = gc * gc * gc;
  const int x = cellp % gp, y = (cellp / gp) % gp, z = cellp / ((int64_t)gp * gp);
  for (int i = threadIdx.x; i < 2 * O * O; i += blockDim.x) se1[i] = e1[i];
  double2 acc[(N + 127) / 128];
#pragma unroll
  for (int i = 0; i < (N + 127) / 128; ++i) acc[i] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int oct = 0; oct < 8; ++oct) {
    const int64_t cc = (2 * x + (oct & 1)) + gc * ((2 * y + ((oct >> 1) & 1)) + gc * (2 * z + (oct >> 2)));
    const double2 *src = cmom + ((int64_t)cs * ncc + cc) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      double2 v = src[k];
      if (phase) v = cmulc(v, phase[((int64_t)oct * nslot_p + slot) * N + k]);
      u[k] = v;
    }
    __syncthreads();
    tensor_transfer<O>(se1, oct, true, u, t);
#pragma unroll
    for (int i = 0; i < (N + 127) / 128; ++i) {
      const int k = threadIdx.x + 128 * i;
      if (k < N) {
        acc[i].x += u[k].x;
        acc[i].y += u[k].y;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < (N + 127) / 128; ++i) {
    const int k = threadIdx.x + 128 * i;
    if (k < N) pmom[((int64_t)slot * ncp + cellp) * N + k] = acc[i];
  }
  (void)nslot_c;
}

// L2L into child slot cs for all parent slots whose direction maps to it.
template <int O>
__global__ void __launch_bounds__(128) k_l2l_fp64(
    const double2 *ploc, double2 *cloc, int gc, const int32_t *pslots,
    const int32_t *pslot_off, const double2 *phase, int nslot_p,
    const double *e1) {
  constexpr int N = O * O * O;
  __shared__ double2 u[N], t[N];
  __shared__ double se1[2 * O * O];
  const int64_t cellc = blockIdx.x;
  const int cs = blockIdx.y;
  const int gp = gc / 2;
  const int64_t ncp = (int64_t)gp * gp * gp, ncc = (int64_t)gc * gc * gc;
  const int x = cellc % gc, y = (cellc / gc) % gc, z = cellc / ((int64_t)gc * gc);
  const int oct = (x & 1) + 2 * (y & 1) + 4 * (z & 1);
  const int64_t cellp = (x >> 1) + (int64_t)gp * ((y >> 1) + (int64_t)gp * (z >> 1));
  for (int i = threadIdx.x; i < 2 * O * O; i += blockDim.x) se1[i] = e1[i];
  double2 acc[(N + 127) / 128];
#pragma unroll
  for (int i = 0; i < (N + 127) / 128; ++i) acc[i] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int q = pslot_off[cs]; q < pslot_off[cs + 1]; ++q) {
    const int ps = pslots[q];
    const double2 *src = ploc + ((int64_t)ps * ncp + cellp) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) u[k] = src[k];
    __syncthreads();
    tensor_transfer<O>(se1, oct, false, u, t);
#pragma unroll
    for (int i = 0; i < (N + 127) / 128; ++i) {
      const int k = threadIdx.x + 128 * i;
      if (k < N) {
        double2 v = u[k];
        if (phase) v = cmul(v, phase[((int64_t)oct * nslot_p + ps) * N + k]);
        acc[i].x += v.x;
        acc[i].y += v.y;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < (N + 127) / 128; ++i) {
    const int k = threadIdx.x + 128 * i;
    if (k < N) {
      double2 *dst = cloc + ((int64_t)cs * ncc + cellc) * N + k;
      double2 v = *dst;
      v.x += acc[i].x;
      v.y += acc[i].y;
      *dst = v;
    }
  }
}

// ------------------------------------------------------------- M2L (FP64)
// One block: 32 targets of parity alpha in a row of the parent grid, all N
// outputs (warp w takes outputs w, w + 16, ...); loops over the level's
// operators for alpha (sorted by direction slot), accumulating in registers
// and flushing when the slot changes.  Each complex multiply-add is four
// FP64 FMAs; sixteen warps keep the FP64 pipes of the SM busy.
constexpr int kM2lKc = 8;
constexpr int kM2lJG = 16;                  // warps per block

template <int O>
__global__ void __launch_bounds__(kM2lJG * 32, 1) k_m2l_fp64(
    const double2 *ops, const int32_t *alpha_ops, const int32_t *alpha_off,
    const int32_t *op_off, const int32_t *op_slot, const double2 *mom,
    double2 *loc, int g) {
  constexpr int N = O * O * O;
  constexpr int JG = kM2lJG;
  constexpr int NJ = (N + JG - 1) / JG;
  __shared__ double2 sA[N][kM2lKc];
  __shared__ double2 sV[kM2lKc][32];
  const int gp = g >> 1;
  // the block's 32 targets: a bx x by x bz box of the parent grid (all 32
  // lanes carry a target on grids of at least 32 cells in all)
  const int bx = min(gp, 32), by = min(gp, 32 / bx), bz = 32 / (bx * by);
  const int tiles_x = (gp + bx - 1) / bx, tiles_y = (gp + by - 1) / by;
  const int alpha = blockIdx.y;
  const int tile = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int X = (tile % tiles_x) * bx + lane % bx;
  const int Y = ((tile / tiles_x) % tiles_y) * by + (lane / bx) % by;
  const int Z = (tile / (tiles_x * tiles_y)) * bz + lane / (bx * by);
  const int ax = alpha & 1, ay = (alpha >> 1) & 1, az = (alpha >> 2) & 1;
  const int64_t ncell = (int64_t)g * g * g;
  const int tx = 2 * X + ax, ty = 2 * Y + ay, tz = 2 * Z + az;
  const bool tvalid = X < gp && Y < gp && Z < gp;
  const int64_t tcell = tx + (int64_t)g * (ty + (int64_t)g * tz);
  double2 acc[NJ];
#pragma unroll
  for (int i = 0; i < NJ; ++i) acc[i] = make_double2(0.0, 0.0);
  int cur = -1;
  const int i0 = alpha_off[alpha], i1 = alpha_off[alpha + 1];
  for (int ii = i0; ii <= i1; ++ii) {
    const int op = (ii < i1) ? alpha_ops[ii] : -1;
    const int slot = (op >= 0) ? op_slot[op] : -1;
    if (slot != cur) {
      if (cur >= 0 && tvalid) {
#pragma unroll
        for (int i = 0; i < NJ; ++i) {
          const int j = warp + JG * i;
          if (j < N) {
            double2 *dst = loc + ((int64_t)cur * ncell + tcell) * N + j;
            double2 v = *dst;
            v.x += acc[i].x;
            v.y += acc[i].y;
            *dst = v;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < NJ; ++i) acc[i] = make_double2(0.0, 0.0);
      cur = slot;
    }
    if (op < 0) break;
    const int sx = tx - op_off[3 * op], sy = ty - op_off[3 * op + 1], sz = tz - op_off[3 * op + 2];
    const bool svalid = tvalid && sx >= 0 && sy >= 0 && sz >= 0 && sx < g && sy < g && sz < g;
    const double2 *src = mom + ((int64_t)slot * ncell + (svalid ? (sx + (int64_t)g * (sy + (int64_t)g * sz)) : 0)) * N;
    const double2 *A = ops + (int64_t)op * N * N;
    for (int k0 = 0; k0 < N; k0 += kM2lKc) {
      __syncthreads();
      for (int e = threadIdx.x; e < N * kM2lKc; e += blockDim.x) {
        const int j = e / kM2lKc, kk = e % kM2lKc;
        sA[j][kk] = (k0 + kk < N) ? A[(int64_t)j * N + k0 + kk] : make_double2(0.0, 0.0);
      }
      if (warp < kM2lKc) {
        const int k = k0 + warp;
        sV[warp][lane] = (svalid && k < N) ? src[k] : make_double2(0.0, 0.0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kM2lKc; ++kk) {
        const double2 v = sV[kk][lane];
#pragma unroll
        for (int i = 0; i < NJ; ++i) {
          const int j = warp + JG * i;
          if (j < N) {
            const double2 a = sA[j][kk];
            acc[i].x = fma(a.x, v.x, acc[i].x);
            acc[i].x = fma(-a.y, v.y, acc[i].x);
            acc[i].y = fma(a.x, v.y, acc[i].y);
            acc[i].y = fma(a.y, v.x, acc[i].y);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------- L2T (FP64)
template <int O>
__global__ void __launch_bounds__(128) k_l2t_fp64(
    const double *xyz, int64_t n_pts, const int32_t *leaf_cell,
    const int32_t *leaf_begin, const int32_t *leaf_end, double lo0, double lo1,
    double lo2, double w, int g, const double *dir, int nslots, double kappa,
    const double2 *loc, int64_t ncell, double2 *ysorted) {
  constexpr int N = O * O * O;
  __shared__ double2 sg[N];
  __shared__ double2 red[4];
  const int leaf = blockIdx.x;
  const int cell = leaf_cell[leaf];
  const int cx = cell % g, cy = (cell / g) % g, cz = cell / (g * g);
  const double m0 = lo0 + (cx + 0.5) * w, m1 = lo1 + (cy + 0.5) * w, m2 = lo2 + (cz + 0.5) * w;
  const double inv_h = 2.0 / w;
  const int b = leaf_begin[leaf], e = leaf_end[leaf];
  for (int p = b; p < e; ++p) {
    const double y0 = xyz[p] - m0, y1 = xyz[n_pts + p] - m1, y2 = xyz[2 * n_pts + p] - m2;
    double lx[O], ly[O], lz[O];
    lagrange1d<O>(y0 * inv_h, lx);
    lagrange1d<O>(y1 * inv_h, ly);
    lagrange1d<O>(y2 * inv_h, lz);
    double2 tot = make_double2(0.0, 0.0);
    for (int slot = 0; slot < nslots; ++slot) {
      const double2 *src = loc + ((int64_t)slot * ncell + cell) * N;
      double2 s = make_double2(0.0, 0.0);
      for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int kx = k % O, ky = (k / O) % O, kz = k / (O * O);
        const double l = lx[kx] * ly[ky] * lz[kz];
        const double2 v = src[k];
        s.x += l * v.x;
        s.y += l * v.y;
      }
      const double2 ph = cexpi(kappa * (y0 * dir[3 * slot] + y1 * dir[3 * slot + 1] + y2 * dir[3 * slot + 2]));
      const double2 t = cmul(s, ph);
      tot.x += t.x;
      tot.y += t.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      tot.x += __shfl_down_sync(0xffffffffu, tot.x, o);
      tot.y += __shfl_down_sync(0xffffffffu, tot.y, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
      double2 r = red[0];
      for (int i = 1; i < 4; ++i) {
        r.x += red[i].x;
        r.y += red[i].y;
      }
      ysorted[p] = r;
    }
    __syncthreads();
  }
  (void)sg;
}

// ---------------------------------------------------- nearfield (FP64)
// One thread per target point; sources of every nearfield leaf read in order.
__global__ void __launch_bounds__(128) k_p2p_fp64(
    const double *txyz, int64_t nt, const int32_t *tperm, const int32_t *leaf_cell,
    const int32_t *leaf_begin, const int32_t *leaf_end, const double *sxyz,
    int64_t ns, const int32_t *sperm, const int32_t *s_leaf_of_cell,
    const int32_t *sb, const int32_t *se, int g, const int32_t *near_off, int nnear,
    double kappa, const double2 *x, const double2 *ysorted, double2 *y) {
  const int leaf = blockIdx.x;
  const int cell = leaf_cell[leaf];
  const int cx = cell % g, cy = (cell / g) % g, cz = cell / (g * g);
  const int b = leaf_begin[leaf], e = leaf_end[leaf];
  const double inv4pi = 1.0 / (4.0 * kPi);
  for (int p = b + threadIdx.x; p < e; p += blockDim.x) {
    const double x0 = txyz[p], x1 = txyz[nt + p], x2 = txyz[2 * nt + p];
    double2 acc = ysorted[p];
    for (int i = 0; i < nnear; ++i) {
      const int sx = cx - near_off[3 * i], sy = cy - near_off[3 * i + 1], sz = cz - near_off[3 * i + 2];
      if (sx < 0 || sy < 0 || sz < 0 || sx >= g || sy >= g || sz >= g) continue;
      const int s = s_leaf_of_cell[sx + g * (sy + g * sz)];
      if (s < 0) continue;
      for (int q = sb[s]; q < se[s]; ++q) {
        const double y0 = sxyz[q], y1 = sxyz[ns + q], y2 = sxyz[2 * ns + q];
        if (x0 == y0 && x1 == y1 && x2 == y2) continue;   // zero diagonal
        const double d0 = x0 - y0, d1 = x1 - y1, d2 = x2 - y2;
        const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        const double2 f = cexpi(kappa * r);
        const double sc = inv4pi / r;
        const double2 v = x[sperm[q]];
        acc.x += sc * (f.x * v.x - f.y * v.y);
        acc.y += sc * (f.x * v.y + f.y * v.x);
      }
    }
    y[tperm[p]] = acc;
  }
}

}  // namespace

// ------------------------------------------------------------------ host
void build_operators_fp64(Plan &plan, cudaStream_t st) {
  const int o = plan.order, n = plan.n;
  // reference nodes and barycentric factors (Eq. 4, reading R1)
  double cheb[kMaxOrder] = {0}, lagw[kMaxOrder] = {0};
  chebyshev_tables(o, cheb, lagw);
  DFDM_CUDA_TRY(cudaMemcpyToSymbol(c_cheb, cheb, sizeof(cheb)));
  DFDM_CUDA_TRY(cudaMemcpyToSymbol(c_lagw, lagw, sizeof(lagw)));
  // 1-D transfer matrices: e1[b][k][l] = L_l((2b - 1 + r_k) / 2)
  std::vector<double> e1(2 * o * o);
  for (int b = 0; b < 2; ++b)
    for (int k = 0; k < o; ++k) {
      const double t = (2.0 * b - 1.0 + cheb[k]) / 2.0;
      for (int l = 0; l < o; ++l) {
        double v = lagw[l];
        for (int mu = 0; mu < o; ++mu)
          if (mu != l) v *= (t - cheb[mu]);
        e1[(b * o + k) * o + l] = v;
      }
    }
  plan.e1 = plan.alloc<double>(2 * o * o);
  DFDM_CUDA_TRY(cudaMemcpyAsync(plan.e1, e1.data(), e1.size() * sizeof(double), cudaMemcpyHostToDevice, st));

  // per-operator tables
  const int nops = plan.n_ops;
  std::vector<int32_t> op_level, op_off, op_slot;
  std::vector<double> op_dir, level_w;
  for (auto &L : plan.levels) {
    level_w.push_back(L.w);
    for (size_t i = 0; i < L.op_dir.size(); ++i) {
      op_level.push_back(L.level);
      op_off.insert(op_off.end(), L.off.begin() + 3 * i, L.off.begin() + 3 * i + 3);
      op_slot.push_back(L.op_slot[i]);
      double c[3];
      direction_vector(plan.l_hf, L.level, L.op_dir[i], c);
      op_dir.insert(op_dir.end(), c, c + 3);
    }
  }
  plan.op_off_dev = plan.alloc<int32_t>(3 * std::max(nops, 1));
  plan.op_slot_dev = plan.alloc<int32_t>(std::max(nops, 1));
  if (nops > 0) {
    DFDM_CUDA_TRY(cudaMemcpyAsync(plan.op_off_dev, op_off.data(), op_off.size() * 4, cudaMemcpyHostToDevice, st));
    DFDM_CUDA_TRY(cudaMemcpyAsync(plan.op_slot_dev, op_slot.data(), op_slot.size() * 4, cudaMemcpyHostToDevice, st));
  }
  if (plan.params.precision == DFDM_FP64 && nops > 0) {
    int32_t *d_level = nullptr;
    double *d_dir = nullptr, *d_w = nullptr;
    DFDM_CUDA_TRY(cudaMalloc(&d_level, nops * 4));
    DFDM_CUDA_TRY(cudaMalloc(&d_dir, nops * 3 * 8));
    DFDM_CUDA_TRY(cudaMalloc(&d_w, level_w.size() * 8));
    DFDM_CUDA_TRY(cudaMemcpyAsync(d_level, op_level.data(), nops * 4, cudaMemcpyHostToDevice, st));
    DFDM_CUDA_TRY(cudaMemcpyAsync(d_dir, op_dir.data(), nops * 3 * 8, cudaMemcpyHostToDevice, st));
    DFDM_CUDA_TRY(cudaMemcpyAsync(d_w, level_w.data(), level_w.size() * 8, cudaMemcpyHostToDevice, st));
    plan.coupling = plan.alloc<double2>((size_t)nops * n * n);
    dim3 grid(nops, n);
    k_coupling_fp64<<<grid, 128, 0, st>>>(o, n, d_level, plan.op_off_dev, d_dir, d_w, plan.kappa, plan.coupling);
    DFDM_LAUNCH_CHECK();
    DFDM_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(d_level);
    cudaFree(d_dir);
    cudaFree(d_w);
  }

  // M2L worklists, child slot maps, direction vectors, nearfield offsets
  std::vector<int32_t> ops_all, child_all;
  plan.m2l_ops_off.assign((plan.depth + 1) * 9, 0);
  plan.child_slot_off.assign(plan.depth + 2, 0);
  plan.dir_vec_off.assign(plan.depth + 2, 0);
  std::vector<double> dirs_all;
  for (auto &L : plan.levels) {
    for (int a = 0; a < 8; ++a) {
      plan.m2l_ops_off[L.level * 9 + a] = (int64_t)ops_all.size();
      for (int op : L.alpha_ops[a]) ops_all.push_back(L.op_base + op);
    }
    plan.m2l_ops_off[L.level * 9 + 8] = (int64_t)ops_all.size();
    plan.child_slot_off[L.level] = (int64_t)child_all.size();
    child_all.insert(child_all.end(), L.child_slot.begin(), L.child_slot.end());
    plan.dir_vec_off[L.level] = (int64_t)dirs_all.size();
    dirs_all.insert(dirs_all.end(), L.dir_vec.begin(), L.dir_vec.end());
  }
  plan.child_slot_off[plan.depth + 1] = (int64_t)child_all.size();
  plan.dir_vec_off[plan.depth + 1] = (int64_t)dirs_all.size();
  plan.m2l_ops = plan.alloc<int32_t>(std::max<size_t>(ops_all.size(), 1));
  plan.child_slot_dev = plan.alloc<int32_t>(std::max<size_t>(child_all.size(), 1));
  plan.dir_vec_dev = plan.alloc<double>(std::max<size_t>(dirs_all.size(), 1));
  plan.near_off_dev = plan.alloc<int32_t>(std::max<size_t>(plan.near_off.size(), 1));
  if (!ops_all.empty())
    DFDM_CUDA_TRY(cudaMemcpyAsync(plan.m2l_ops, ops_all.data(), ops_all.size() * 4, cudaMemcpyHostToDevice, st));
  if (!child_all.empty())
    DFDM_CUDA_TRY(cudaMemcpyAsync(plan.child_slot_dev, child_all.data(), child_all.size() * 4, cudaMemcpyHostToDevice, st));
  if (!dirs_all.empty())
    DFDM_CUDA_TRY(cudaMemcpyAsync(plan.dir_vec_dev, dirs_all.data(), dirs_all.size() * 8, cudaMemcpyHostToDevice, st));
  DFDM_CUDA_TRY(cudaMemcpyAsync(plan.near_off_dev, plan.near_off.data(), plan.near_off.size() * 4, cudaMemcpyHostToDevice, st));

  // per-level alpha offsets (relative to the level's list) and, for L2L, the
  // parent slots mapping to each child slot
  {
    std::vector<int32_t> aoff((plan.depth + 1) * 9, 0);
    for (int l = 0; l <= plan.depth; ++l)
      for (int a = 0; a < 9; ++a)
        aoff[l * 9 + a] = (int32_t)(plan.m2l_ops_off[l * 9 + a] - plan.m2l_ops_off[l * 9]);
    plan.m2l_aoff_dev = plan.alloc<int32_t>(aoff.size());
    DFDM_CUDA_TRY(cudaMemcpyAsync(plan.m2l_aoff_dev, aoff.data(), aoff.size() * 4, cudaMemcpyHostToDevice, st));
    std::vector<int32_t> ps_all, po_all;
    plan.l2l_pslots_off.assign(plan.depth + 1, 0);
    plan.l2l_poff_off.assign(plan.depth + 1, 0);
    for (int l = 0; l < plan.depth; ++l) {
      const LevelPlan &L = plan.levels[l];
      const int nsc = (int)plan.levels[l + 1].slot_dir.size();
      plan.l2l_pslots_off[l] = (int64_t)ps_all.size();
      plan.l2l_poff_off[l] = (int64_t)po_all.size();
      int32_t base = 0;
      for (int cs = 0; cs < nsc; ++cs) {
        po_all.push_back(base);
        for (int ps = 0; ps < (int)L.slot_dir.size(); ++ps)
          if (L.child_slot[ps] == cs) {
            ps_all.push_back(ps);
            ++base;
          }
      }
      po_all.push_back(base);
    }
    plan.l2l_pslots_dev = plan.alloc<int32_t>(std::max<size_t>(ps_all.size(), 1));
    plan.l2l_poff_dev = plan.alloc<int32_t>(std::max<size_t>(po_all.size(), 1));
    if (!ps_all.empty())
      DFDM_CUDA_TRY(cudaMemcpyAsync(plan.l2l_pslots_dev, ps_all.data(), ps_all.size() * 4, cudaMemcpyHostToDevice, st));
    if (!po_all.empty())
      DFDM_CUDA_TRY(cudaMemcpyAsync(plan.l2l_poff_dev, po_all.data(), po_all.size() * 4, cudaMemcpyHostToDevice, st));
  }

  // centred directional diagonals for every high-frequency parent level
  plan.m2m_phase_off.assign(plan.depth + 1, -1);
  int64_t total = 0;
  for (int l = plan.min_level; l < plan.depth; ++l) {
    if (!plan.levels[l].high_freq || plan.levels[l].slot_dir.empty()) continue;
    plan.m2m_phase_off[l] = total;
    total += 8ll * (int64_t)plan.levels[l].slot_dir.size() * n;
  }
  if (total > 0) {
    plan.m2m_phase = plan.alloc<double2>(total);
    for (int l = plan.min_level; l < plan.depth; ++l) {
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
      DFDM_CUDA_TRY(cudaMemcpyAsync(d_c, L.dir_vec.data(), 3 * ns * 8, cudaMemcpyHostToDevice, st));
      DFDM_CUDA_TRY(cudaMemcpyAsync(d_c2, c2.data(), 3 * ns * 8, cudaMemcpyHostToDevice, st));
      dim3 grid(ns, 8);
      k_phase_table<<<grid, 128, 0, st>>>(o, n, ns, d_c, d_c2, plan.kappa, 0.25 * L.w,
                                          plan.m2m_phase + plan.m2m_phase_off[l]);
      DFDM_LAUNCH_CHECK();
      DFDM_CUDA_TRY(cudaStreamSynchronize(st));
      cudaFree(d_c);
      cudaFree(d_c2);
    }
  }
  DFDM_CUDA_TRY(cudaStreamSynchronize(st));
}

void count_pairs(Plan &plan, cudaStream_t st) {
  const int p = plan.depth;
  std::vector<uint8_t *> ext(p + 1, nullptr), exs(p + 1, nullptr);
  for (int l = p; l >= 0; --l) {
    const int64_t nc = 1ll << (3 * l);
    DFDM_CUDA_TRY(cudaMalloc(&ext[l], nc));
    DFDM_CUDA_TRY(cudaMalloc(&exs[l], nc));
    if (l == p) {
      k_exist_leaf<<<nblk(nc, 256), 256, 0, st>>>(plan.tt.leaf_of_cell, nc, ext[l]);
      k_exist_leaf<<<nblk(nc, 256), 256, 0, st>>>(plan.ts.leaf_of_cell, nc, exs[l]);
    } else {
      k_exist_up<<<nblk(nc, 256), 256, 0, st>>>(ext[l + 1], 1 << l, ext[l]);
      k_exist_up<<<nblk(nc, 256), 256, 0, st>>>(exs[l + 1], 1 << l, exs[l]);
    }
    DFDM_LAUNCH_CHECK();
  }
  unsigned long long *cnt = nullptr;
  DFDM_CUDA_TRY(cudaMalloc(&cnt, 3 * sizeof(unsigned long long)));
  int64_t total = 0;
  for (int l = 1; l <= p; ++l) {
    DFDM_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
    const int64_t nc = 1ll << (3 * l);
    std::vector<int32_t> aoff(9);
    for (int a = 0; a < 9; ++a)
      aoff[a] = (int32_t)(plan.m2l_ops_off[l * 9 + a] - plan.m2l_ops_off[l * 9]);
    int32_t *d_aoff = nullptr;
    DFDM_CUDA_TRY(cudaMalloc(&d_aoff, 9 * 4));
    DFDM_CUDA_TRY(cudaMemcpyAsync(d_aoff, aoff.data(), 36, cudaMemcpyHostToDevice, st));
    k_count_level<<<nblk(nc, 256), 256, 0, st>>>(ext[l], exs[l], 1 << l, plan.m2l_ops + plan.m2l_ops_off[l * 9],
                                                 d_aoff, plan.op_off_dev, cnt);
    DFDM_LAUNCH_CHECK();
    unsigned long long h = 0;
    DFDM_CUDA_TRY(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
    DFDM_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(d_aoff);
    plan.levels[l].n_coupling = (int64_t)h;
    total += (int64_t)h;
  }
  plan.stats.n_coupling = total;
  DFDM_CUDA_TRY(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st));
  k_count_near<<<nblk(plan.tt.nleaves, 128), 128, 0, st>>>(
      plan.tt.leaf_cell, plan.tt.leaf_begin, plan.tt.leaf_end, plan.tt.nleaves, plan.ts.leaf_of_cell,
      plan.ts.leaf_begin, plan.ts.leaf_end, 1 << p, plan.near_off_dev, (int)(plan.near_off.size() / 3), cnt);
  DFDM_LAUNCH_CHECK();
  unsigned long long h2[2];
  DFDM_CUDA_TRY(cudaMemcpyAsync(h2, cnt, sizeof(h2), cudaMemcpyDeviceToHost, st));
  DFDM_CUDA_TRY(cudaStreamSynchronize(st));
  plan.stats.n_near_blocks = (int64_t)h2[0];
  plan.stats.nf_entries = (int64_t)h2[1];
  cudaFree(cnt);
  for (int l = 0; l <= p; ++l) {
    cudaFree(ext[l]);
    cudaFree(exs[l]);
  }
}

// -------------------------------------------------------------- apply
template <int O>
static void apply_fp64_o(Plan &plan, const double2 *x, double2 *y, cudaStream_t st) {
  constexpr int N = O * O * O;
  const int p = plan.depth;
  const Tree &tt = plan.tt, &ts = plan.ts;
  const double *lo = plan.root_lo;
  double2 *ysorted = plan.ysorted;   // far-field values in sorted target order
  const bool far = plan.min_level <= p;
  if (far) {
    for (int l = plan.min_level; l <= p; ++l) {
      const int64_t nc = 1ll << (3 * l);
      const size_t bytes = (size_t)plan.levels[l].slot_dir.size() * nc * N * sizeof(double2);
      DFDM_CUDA_TRY(cudaMemsetAsync(plan.mom[l], 0, bytes, st));
      DFDM_CUDA_TRY(cudaMemsetAsync(plan.loc[l], 0, bytes, st));
    }
    // S2M on the leaf level
    const LevelPlan &P = plan.levels[p];
    const int nsl = (int)P.slot_dir.size();
    if (nsl > 0 && ts.nleaves > 0) {
      dim3 grid((unsigned)ts.nleaves, nsl);
      k_s2m_fp64<O><<<grid, 128, 0, st>>>(ts.xyz, ts.n, ts.perm, x, ts.leaf_cell, ts.leaf_begin, ts.leaf_end,
                                          lo[0], lo[1], lo[2], P.w, P.grid, plan.dir_vec_dev + plan.dir_vec_off[p],
                                          plan.kappa, plan.mom[p], 1ll << (3 * p));
      DFDM_COUNT_LAUNCH(plan);
    }
    // M2M, levels p-1 .. min_level
    for (int l = p - 1; l >= plan.min_level; --l) {
      const LevelPlan &L = plan.levels[l];
      const int ns = (int)L.slot_dir.size();
      if (ns == 0) continue;
      const double2 *ph = plan.m2m_phase_off[l] >= 0 ? plan.m2m_phase + plan.m2m_phase_off[l] : nullptr;
      dim3 grid((unsigned)(1ll << (3 * l)), ns);
      k_m2m_fp64<O><<<grid, 128, 0, st>>>(plan.mom[l + 1], plan.mom[l], L.grid,
                                          plan.child_slot_dev + plan.child_slot_off[l],
                                          (int)plan.levels[l + 1].slot_dir.size(), ph, ns, plan.e1);
      DFDM_COUNT_LAUNCH(plan);
    }
    // M2L on every level
    for (int l = std::max(1, plan.min_level); l <= p; ++l) {
      const LevelPlan &L = plan.levels[l];
      if (L.off.empty()) continue;
      const int gp = L.grid / 2;
      const int bx = std::min(gp, 32), by = std::min(gp, 32 / bx), bz = 32 / (bx * by);
      const int tiles = ((gp + bx - 1) / bx) * ((gp + by - 1) / by) * ((gp + bz - 1) / bz);
      dim3 grid(tiles, 8);
      PhaseScope sc(plan.timing, kPhM2L0 + l, st);
      k_m2l_fp64<O><<<grid, kM2lJG * 32, 0, st>>>(plan.coupling, plan.m2l_ops + plan.m2l_ops_off[l * 9],
                                          plan.m2l_aoff_dev + 9 * l,
                                          plan.op_off_dev, plan.op_slot_dev, plan.mom[l], plan.loc[l], L.grid);
      DFDM_COUNT_LAUNCH(plan);
    }
    // L2L, levels min_level .. p-1 (into the child level)
    for (int l = plan.min_level; l < p; ++l) {
      const LevelPlan &L = plan.levels[l];
      const LevelPlan &C = plan.levels[l + 1];
      const int nsp = (int)L.slot_dir.size();
      const int nsc = (int)C.slot_dir.size();
      if (nsp == 0 || nsc == 0) continue;
      const int32_t *d_ps = plan.l2l_pslots_dev + plan.l2l_pslots_off[l];
      const int32_t *d_po = plan.l2l_poff_dev + plan.l2l_poff_off[l];
      const double2 *ph = plan.m2m_phase_off[l] >= 0 ? plan.m2m_phase + plan.m2m_phase_off[l] : nullptr;
      dim3 grid((unsigned)(1ll << (3 * (l + 1))), nsc);
      k_l2l_fp64<O><<<grid, 128, 0, st>>>(plan.loc[l], plan.loc[l + 1], C.grid, d_ps, d_po, ph, nsp, plan.e1);
      DFDM_COUNT_LAUNCH(plan);
    }
    // L2T
    const int nslt = (int)P.slot_dir.size();
    if (nslt > 0 && tt.nleaves > 0) {
      k_l2t_fp64<O><<<(unsigned)tt.nleaves, 128, 0, st>>>(
          tt.xyz, tt.n, tt.leaf_cell, tt.leaf_begin, tt.leaf_end, lo[0], lo[1], lo[2], P.w, P.grid,
          plan.dir_vec_dev + plan.dir_vec_off[p], nslt, plan.kappa, plan.loc[p], 1ll << (3 * p), ysorted);
      DFDM_COUNT_LAUNCH(plan);
    } else {
      DFDM_CUDA_TRY(cudaMemsetAsync(ysorted, 0, tt.n * sizeof(double2), st));
    }
  } else {
    DFDM_CUDA_TRY(cudaMemsetAsync(ysorted, 0, tt.n * sizeof(double2), st));
  }
  // nearfield, writing y in the caller's order
  k_p2p_fp64<<<(unsigned)tt.nleaves, 128, 0, st>>>(
      tt.xyz, tt.n, tt.perm, tt.leaf_cell, tt.leaf_begin, tt.leaf_end, ts.xyz, ts.n, ts.perm,
      ts.leaf_of_cell, ts.leaf_begin, ts.leaf_end, 1 << p, plan.near_off_dev, (int)(plan.near_off.size() / 3),
      plan.kappa, x, ysorted, y);
  DFDM_COUNT_LAUNCH(plan);
}

void apply_fp64(Plan &plan, const double2 *x, double2 *y, int nrhs, cudaStream_t st) {
  for (int r = 0; r < nrhs; ++r) {
    const double2 *xr = x + (int64_t)r * plan.ts.n;
    double2 *yr = y + (int64_t)r * plan.tt.n;
    switch (plan.order) {
      case 2: apply_fp64_o<2>(plan, xr, yr, st); break;
      case 3: apply_fp64_o<3>(plan, xr, yr, st); break;
      case 4: apply_fp64_o<4>(plan, xr, yr, st); break;
      case 5: apply_fp64_o<5>(plan, xr, yr, st); break;
      case 6: apply_fp64_o<6>(plan, xr, yr, st); break;
      case 7: apply_fp64_o<7>(plan, xr, yr, st); break;
      default:
        throw Error{DFDM_ERR_UNSUPPORTED, "FP64 form supports orders 2..7"};
    }
  }
}

}  // namespace dfdm
