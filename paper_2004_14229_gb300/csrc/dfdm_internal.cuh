// Internal declarations shared by the library's translation units.
// Fast directional matrix-vector product (Of & Watschinger), GB300 (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dfdm.h"

namespace dfdm {

constexpr int kMaxOrder = 10;
constexpr int kMaxDepth = 10;
constexpr int kMaxLevels = 16;

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
const char *last_error();

struct Error {
  dfdm_status status;
  std::string msg;
};

#define DFDM_CUDA_TRY(expr)                                                  \
  do {                                                                       \
    cudaError_t e_ = (expr);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      throw ::dfdm::Error{e_ == cudaErrorMemoryAllocation ? DFDM_ERR_OOM     \
                                                          : DFDM_ERR_CUDA,   \
                          std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
    }                                                                        \
  } while (0)

#define DFDM_LAUNCH_CHECK() DFDM_CUDA_TRY(cudaGetLastError())
// Checks a launch of an apply and counts it for dfdm_plan_timing.
#define DFDM_COUNT_LAUNCH(plan) \
  do {                          \
    DFDM_LAUNCH_CHECK();        \
    ++(plan).timing.launches;   \
  } while (0)

// ------------------------------------------------------- device buffers
// Owning device allocation; freed by the plan.
struct DevBuf {
  void *ptr = nullptr;
  size_t bytes = 0;
};

// ------------------------------------------------------------------ tree
// One uniform box cluster tree (Alg. 1) on the device, in Morton order.
struct Tree {
  int64_t n = 0;            // points
  int depth = 0;            // p (all leaves on level p)
  int key_depth = 0;        // depth D of the Morton keys
  uint64_t *keys = nullptr; // sorted Morton keys at depth D (n)
  int32_t *perm = nullptr;  // sorted position -> original index (n)
  double *xyz = nullptr;    // sorted coordinates, SoA: x[n], y[n], z[n]
  // non-empty leaves (level p), ascending key
  int64_t nleaves = 0;
  int32_t *leaf_cell = nullptr;  // linear cell index x + G y + G^2 z, G = 2^p
  int32_t *leaf_begin = nullptr; // [begin, end) in sorted order
  int32_t *leaf_end = nullptr;
  int32_t *leaf_of_cell = nullptr; // G^3 lookup: leaf index or -1
  int32_t max_leaf_size = 0;
};

// --------------------------------------------------------------- planner
// Coupling structure of one level (Alg. 2 / Def. 2 on uniform trees) and
// the direction slots of the level (a level-wide superset of Def. 5's sets).
struct LevelPlan {
  int level = 0;
  double w = 0;                 // box side
  int grid = 1;                 // 2^level
  bool high_freq = false;       // level <= l_hf
  int ndir_full = 1;            // |D^(l)|
  std::vector<int> slot_dir;    // slot -> index in D^(l)
  std::vector<int> dir_slot;    // index in D^(l) -> slot, -1 unused
  std::vector<double> dir_vec;  // slot -> unit vector (3 doubles), 0 on LF
  std::vector<int> child_slot;  // slot -> slot of dir_(l+1)(c) on level l+1
  // distinct admissible offsets (one stored coupling matrix each)
  std::vector<int> off;         // 3 ints per operator
  std::vector<int> op_dir;      // index in D^(l) of c(d)
  std::vector<int> op_slot;     // slot of c(d)
  int op_base = 0;              // index of this level's first operator
  // per parity alpha: operator list sorted by slot
  std::vector<int> alpha_ops[8];
  int64_t n_coupling = 0;       // N_C on this level (non-empty pairs)
};

struct TcState;  // tensor-core form's tables (tc.cu)

// Per-phase CUDA-event timing of an apply (dfdm_plan_set_timing).
enum Phase { kPhS2M = 0, kPhM2M, kPhSplit, kPhL2L, kPhL2T, kPhNear, kPhM2L0 };
struct Timing {
  bool on = false;
  bool valid = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Seg {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Seg> segs;
  int64_t launches = 0;       // kernel launches of the last apply
  int64_t acc_launches = 0;   // launches of the applies since timing was turned on or read
  int64_t applies = 0;        // applies whose segments are held
  cudaEvent_t next() {
    if (used == pool.size()) {
      cudaEvent_t e;
      DFDM_CUDA_TRY(cudaEventCreate(&e));
      pool.push_back(e);
    }
    return pool[used++];
  }
  void reset() {
    used = 0;
    segs.clear();
    acc_launches = 0;
    applies = 0;
    valid = false;
  }
  void destroy() {
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
    used = 0;
  }
};

// Records events around one phase when timing is on.
struct PhaseScope {
  Timing &t;
  int phase;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  PhaseScope(Timing &t_, int ph, cudaStream_t s) : t(t_), phase(ph), st(s) {
    if (t.on) {
      a = t.next();
      DFDM_CUDA_TRY(cudaEventRecord(a, st));
    }
  }
  ~PhaseScope() noexcept(false) {
    if (t.on && a) {
      cudaEvent_t b = t.next();
      DFDM_CUDA_TRY(cudaEventRecord(b, st));
      t.segs.push_back(Timing::Seg{phase, a, b});
    }
  }
};

struct Plan {
  dfdm_params params{};
  double kappa = 0;
  int order = 0, n = 0;         // nodes per axis, nodes per box
  double root_lo[3] = {0, 0, 0};
  double root_side = 1;
  int depth = 0;
  int l_hf = -1;
  int min_level = 1;            // coarsest level with moments
  Tree tt, ts;
  std::vector<LevelPlan> levels;
  std::vector<int> near_off;    // 3 ints per nearfield offset on level p
  int n_ops = 0;
  dfdm_stats stats{};

  // device tables
  double *cheb = nullptr;               // o reference nodes
  double2 *coupling = nullptr;          // FP64 coupling operators [op][j][k]
  double *e1 = nullptr;                 // 1-D transfer matrices [2][o][o]
  double2 *m2m_phase = nullptr;         // [level][oct][slot][n] (HF parents)
  std::vector<int64_t> m2m_phase_off;   // per level offset into m2m_phase
  double *dir_vec_dev = nullptr;        // slot directions per level, 3 doubles
  std::vector<int64_t> dir_vec_off;
  int32_t *m2l_ops = nullptr;           // [level] per alpha op lists
  std::vector<int64_t> m2l_ops_off;     // per (level, alpha) offset, 9 per level
  int32_t *op_off_dev = nullptr;        // 3 ints per operator
  int32_t *op_slot_dev = nullptr;       // per operator
  int32_t *child_slot_dev = nullptr;    // per level, slot -> child slot
  std::vector<int64_t> child_slot_off;
  int32_t *near_off_dev = nullptr;      // 3 ints per nearfield offset
  int32_t *m2l_aoff_dev = nullptr;      // per level 9 alpha offsets into its op list
  int32_t *l2l_pslots_dev = nullptr;    // per level: parent slots of each child slot
  int32_t *l2l_poff_dev = nullptr;
  std::vector<int64_t> l2l_pslots_off, l2l_poff_off;
  double2 *ysorted = nullptr;           // far-field result in sorted target order
  // moments and locals per level: [slot][cell][n] complex128
  std::vector<double2 *> mom, loc;
  // staging for dfdm_apply_host: pinned host and device buffers
  void *x_stage = nullptr, *y_stage = nullptr;
  void *x_dev_stage = nullptr, *y_dev_stage = nullptr;
  size_t stage_bytes = 0;
  int *err_flag = nullptr;              // device error word
  TcState *tc = nullptr;
  Timing timing;

  std::vector<DevBuf> owned;
  int64_t device_bytes = 0;

  template <typename T>
  T *alloc(size_t count) {
    void *p = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    DFDM_CUDA_TRY(cudaMalloc(&p, bytes));
    owned.push_back(DevBuf{p, bytes});
    device_bytes += (int64_t)bytes;
    return static_cast<T *>(p);
  }
  void free_all();
};

// ------------------------------------------------------- entry points of
// the translation units
// tree.cu
void build_tree(Plan &plan, Tree &tree, const double *host_pts, int64_t n,
                cudaStream_t st);
void export_level(const Plan &plan, const Tree &tree, int level,
                  std::vector<int64_t> &keys, std::vector<int64_t> &begin,
                  std::vector<int64_t> &end, cudaStream_t st);
// planner.cu
void chebyshev_tables(int order, double *cheb, double *lagw);
int default_l_hf(double kappa, double root_side, int p);
void build_levels(Plan &plan);
int face_index(int l_hf, int level, const int d[3]);
void direction_vector(int l_hf, int level, int j, double out[3]);
// direct.cu
// Fixed scratch of dfdm_direct_rows_noalloc: complex128 entries (4 MiB),
// enough for nrows x chunks partial sums with nrows <= this count.
constexpr int64_t kNoAllocScratchEntries = (int64_t)1 << 18;
constexpr int kMaxDevicesNoAlloc = 64;
int direct_chunks(int64_t nrows, int64_t ns);
double2 *noalloc_scratch();
void direct_rows(const double *tgt, int64_t nt, const double *src, int64_t ns, double kappa, const double2 *x,
                 const int64_t *rows, int64_t nrows, double2 *y, double2 *scratch, int nchunk,
                 cudaStream_t st);
// fp64.cu
void build_operators_fp64(Plan &plan, cudaStream_t st);
void count_pairs(Plan &plan, cudaStream_t st);
void apply_fp64(Plan &plan, const double2 *x, double2 *y, int nrhs,
                cudaStream_t st);

}  // namespace dfdm

// The opaque handle of include/dfdm.h.
struct dfdm_plan_s {
  dfdm::Plan p;
};
