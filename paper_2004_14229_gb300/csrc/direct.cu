// Direct evaluation of Eq. (1) at selected target rows (the "direct
// computation" Sect. 4 compares the method with), in FP64 on the GPU.
//
// Few rows against many sources: the sources are split into `nchunk` chunks;
// block (row tile, chunk) forms the partial sums of its rows over its chunk
// in a scratch array partial[chunk][row] (one write per entry, so the scratch
// needs no clearing), and a second kernel adds the chunks in a fixed order.
#include <mutex>

#include "dfdm_internal.cuh"

namespace dfdm {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kRowsPerBlock = 128;
constexpr int kSrcTile = 256;

__global__ void __launch_bounds__(kRowsPerBlock) k_direct_partial(const double *tgt, int64_t nt, const double *src,
                                                                 int64_t ns,
                                                                 double kappa, const double2 *x,
                                                                 const int64_t *rows, int64_t nrows, int nchunk,
                                                                 double2 *partial) {
  __shared__ double3 sp[kSrcTile];
  __shared__ double2 sv[kSrcTile];
  const int64_t r = (int64_t)blockIdx.x * kRowsPerBlock + threadIdx.x;
  const int chunk = blockIdx.y;
  const int64_t per = (ns + nchunk - 1) / nchunk;
  const int64_t k0 = chunk * per, k1 = min(ns, k0 + per);
  const int64_t j = (r < nrows) ? rows[r] : -1;
  const bool act = j >= 0 && j < nt;      // an out-of-range row reads nothing
  double x0 = 0, x1 = 0, x2 = 0;
  if (act) {
    x0 = tgt[3 * j];
    x1 = tgt[3 * j + 1];
    x2 = tgt[3 * j + 2];
  }
  const double inv4pi = 1.0 / (4.0 * kPi);
  double ar = 0.0, ai = 0.0;
  for (int64_t q0 = k0; q0 < k1; q0 += kSrcTile) {
    const int cnt = (int)min((int64_t)kSrcTile, k1 - q0);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const int64_t q = q0 + i;
      sp[i] = make_double3(src[3 * q], src[3 * q + 1], src[3 * q + 2]);
      sv[i] = x[q];
    }
    __syncthreads();
    if (act) {
      for (int i = 0; i < cnt; ++i) {
        const double3 y = sp[i];
        if (x0 == y.x && x1 == y.y && x2 == y.z) continue;   // zero diagonal
        const double d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z;
        const double rr = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        double s, c;
        sincos(kappa * rr, &s, &c);
        const double sc = inv4pi / rr;
        const double2 v = sv[i];
        ar += sc * (c * v.x - s * v.y);
        ai += sc * (c * v.y + s * v.x);
      }
    }
  }
  if (r < nrows) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    partial[(int64_t)chunk * nrows + r] = act ? make_double2(ar, ai) : make_double2(nan, nan);
  }
}

__global__ void k_direct_reduce(const double2 *partial, int64_t nrows, int nchunk, double2 *y) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  double2 s = make_double2(0.0, 0.0);
  for (int c = 0; c < nchunk; ++c) {
    const double2 v = partial[(int64_t)c * nrows + r];
    s.x += v.x;
    s.y += v.y;
  }
  y[r] = s;
}

}  // namespace

int direct_chunks(int64_t nrows, int64_t ns) {
  // enough blocks to fill the GPU several times over
  const int64_t tiles = (nrows + kRowsPerBlock - 1) / kRowsPerBlock;
  int64_t c = (4 * 152 + tiles - 1) / tiles;
  c = std::max<int64_t>(1, std::min<int64_t>(c, 64));
  c = std::min<int64_t>(c, std::max<int64_t>(1, ns / kSrcTile));
  return (int)c;
}

// ------------------------------------------------ fixed scratch (no allocation)
// Scratch of dfdm_direct_rows_noalloc: a file-scope device array that every
// GPU loading the library holds until the process exits.  Host code only
// sees a stand-in symbol for it; the device address comes from
// cudaGetSymbolAddress, once per device, with that device current.
namespace {
__device__ __align__(256) static double2 g_direct_scratch[kNoAllocScratchEntries];
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevicesNoAlloc] = {};
}  // namespace

double2 *noalloc_scratch() {
  int dev = 0;
  DFDM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevicesNoAlloc)
    throw Error{DFDM_ERR_UNSUPPORTED, "device ordinal beyond the no-alloc scratch table"};
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_direct_scratch);
    if (e != cudaSuccess || p == nullptr)
      throw Error{DFDM_ERR_CUDA, std::string("cudaGetSymbolAddress of the fixed scratch failed: ") +
                                     cudaGetErrorString(e)};
    g_scratch_addr[dev] = p;
  }
  return static_cast<double2 *>(g_scratch_addr[dev]);
}

void direct_rows(const double *tgt, int64_t nt, const double *src, int64_t ns, double kappa, const double2 *x,
                 const int64_t *rows, int64_t nrows, double2 *y, double2 *scratch, int nchunk,
                 cudaStream_t st) {
  const unsigned tiles = (unsigned)((nrows + kRowsPerBlock - 1) / kRowsPerBlock);
  k_direct_partial<<<dim3(tiles, nchunk), kRowsPerBlock, 0, st>>>(tgt, nt, src, ns, kappa, x, rows, nrows, nchunk,
                                                                   scratch);
  DFDM_LAUNCH_CHECK();
  k_direct_reduce<<<(unsigned)((nrows + 255) / 256), 256, 0, st>>>(scratch, nrows, nchunk, y);
  DFDM_LAUNCH_CHECK();
}

}  // namespace dfdm
