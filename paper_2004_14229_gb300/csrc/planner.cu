// Host planner: block partition (Alg. 2 / Def. 2), directions (Alg. 3,
// Def. 3) and direction slots (Def. 5) for uniform box cluster trees.
//
// On uniform trees every box of level l is a translate of every other, so
// Alg. 2 reduces to integer box offsets d = t - s on the level-l grid:
//   * the pair (t, s) is admissible iff (A1) and (A3) hold; with box side
//     w, diam = sqrt(3) w and dist = w sqrt(g), g = sum_i max(0, |d_i| - 1)^2,
//     so (A1) <=> 3 <= eta2^2 g and (A3) <=> 9 kappa^2 w^2 <= eta2^2 g, g > 0;
//   * a pair on level l is a node of the block tree iff its parent pair is
//     inadmissible (admissibility is inherited by children: g grows at least
//     4x per level while the (A3) bound shrinks 4x), so the admissible leaves
//     of level l, for a target of parity alpha = t mod 2, have offsets
//     I(l, alpha) = { d : adm_l(d), not adm_{l-1}(ceil((d - alpha) / 2)) };
//   * the inadmissible leaves are the pairs on the leaf level p with
//     not adm_p(d).
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <set>
#include <tuple>

#include "dfdm_internal.cuh"

namespace dfdm {
namespace {

bool admissible(const int d[3], double kappa, double eta2, double w) {
  long long g = 0;
  for (int i = 0; i < 3; ++i) {
    const long long a = std::llabs((long long)d[i]) - 1;
    if (a > 0) g += a * a;
  }
  if (g == 0) return false;
  const double rhs = eta2 * eta2 * (double)g;
  const bool a1 = 3.0 <= rhs;
  const bool a3 = 9.0 * kappa * kappa * w * w <= rhs;
  return a1 && a3;
}

// Largest |d_i| an inadmissible offset can have on a level of box side w:
// inadmissible needs g < max(3, 9 kappa^2 w^2) / eta2^2 (or g = 0).
int near_radius(double kappa, double eta2, double w, int grid) {
  const double thr = std::max(3.0, 9.0 * kappa * kappa * w * w) / (eta2 * eta2);
  const double b = std::floor(std::sqrt(thr)) + 2.0;
  return (int)std::min<double>(b, (double)(grid - 1));
}

inline int floor_div2(int a) { return (a >= 0) ? a / 2 : -((-a + 1) / 2); }

int interleave(int iu, int iv, int r) {
  int j = 0;
  for (int b = 0; b < r; ++b) {
    j |= ((iv >> b) & 1) << (2 * b);
    j |= ((iu >> b) & 1) << (2 * b + 1);
  }
  return j;
}

}  // namespace

// Reference Chebyshev nodes of Eq. (4) (reading: cos((2 nu - 1) pi / (2 (m+1))),
// nu = 1 .. m+1, stored 0-based) and the barycentric factors
// 1 / prod_{mu != nu} (r_nu - r_mu) of their Lagrange polynomials.
void chebyshev_tables(int order, double *cheb, double *lagw) {
  const double pi = 3.14159265358979323846;
  for (int nu = 0; nu < order; ++nu) cheb[nu] = std::cos((2.0 * nu + 1.0) * pi / (2.0 * order));
  for (int nu = 0; nu < order; ++nu) {
    double d = 1.0;
    for (int mu = 0; mu < order; ++mu)
      if (mu != nu) d *= (cheb[nu] - cheb[mu]);
    lagw[nu] = 1.0 / d;
  }
}

int default_l_hf(double kappa, double root_side, int p) {
  int l_hf = -1;
  for (int l = 0; l <= p; ++l)
    if (kappa * std::ldexp(root_side, -l) > 2.0) l_hf = l;
  return l_hf;
}

// j(v) of Def. 3 for a non-zero integer vector on a high-frequency level:
// the first axis attaining max |v_i| (closed faces, smallest index wins), its
// sign, then the sub-face cell along the free axes, a boundary going to the
// lower cell.  Faces -x,+x,-y,+y,-z,+z; free axes in increasing order;
// sub-face 2 h_u + h_v per subdivision, so j = f 4^r + interleave(i_u, i_v).
int face_index(int l_hf, int level, const int d[3]) {
  if (level > l_hf) return 0;
  const int r = l_hf - level;
  int m = 0;
  for (int i = 0; i < 3; ++i) m = std::max(m, std::abs(d[i]));
  int axis = 0;
  while (std::abs(d[axis]) != m) ++axis;
  const int f = 2 * axis + (d[axis] > 0 ? 1 : 0);
  int uv[2], k = 0;
  for (int i = 0; i < 3; ++i)
    if (i != axis) uv[k++] = i;
  int cell[2];
  for (int q = 0; q < 2; ++q) {
    const long long num = (long long)(d[uv[q]] + m) << r;
    const long long den = 2ll * m;
    const long long c = (num + den - 1) / den - 1;   // ceil(num/den) - 1
    cell[q] = (int)std::max(0ll, c);
  }
  return f * (1 << (2 * r)) + interleave(cell[0], cell[1], r);
}

// Normalised midpoint of sub-face j of level `level` (Alg. 3).
void direction_vector(int l_hf, int level, int j, double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  if (level > l_hf) return;
  const int r = l_hf - level;
  const int f = j >> (2 * r);
  const int q = j & ((1 << (2 * r)) - 1);
  int iu = 0, iv = 0;
  for (int b = 0; b < r; ++b) {
    iv |= ((q >> (2 * b)) & 1) << b;
    iu |= ((q >> (2 * b + 1)) & 1) << b;
  }
  const int axis = f / 2;
  double mid[3];
  mid[axis] = (f & 1) ? 1.0 : -1.0;
  int k = 0;
  for (int i = 0; i < 3; ++i) {
    if (i == axis) continue;
    const int c = (k == 0) ? iu : iv;
    mid[i] = -1.0 + std::ldexp(2.0 * c + 1.0, -r);
    ++k;
  }
  const double nrm = std::sqrt(mid[0] * mid[0] + mid[1] * mid[1] + mid[2] * mid[2]);
  for (int i = 0; i < 3; ++i) out[i] = mid[i] / nrm;
}

void build_levels(Plan &plan) {
  const int p = plan.depth;
  const double kappa = plan.kappa, eta2 = plan.params.eta2;
  plan.levels.assign(p + 1, LevelPlan{});
  std::vector<std::set<int>> used(p + 1);
  int op_base = 0;
  for (int l = 0; l <= p; ++l) {
    LevelPlan &L = plan.levels[l];
    L.level = l;
    L.w = std::ldexp(plan.root_side, -l);
    L.grid = 1 << l;
    L.high_freq = (l <= plan.l_hf);
    L.ndir_full = L.high_freq ? 6 * (1 << (2 * (plan.l_hf - l))) : 1;
    if (l == 0) continue;
    // inadmissible parent offsets on level l-1 (bounded by the grid)
    const double wp = std::ldexp(plan.root_side, -(l - 1));
    const int gp = 1 << (l - 1);
    std::set<std::array<int, 3>> parent_near;
    int R = 0;
    // the inadmissible region is bounded: g < 9 kappa^2 wp^2 / eta2^2 + 3/eta2^2
    const int rp = near_radius(kappa, eta2, wp, gp);
    for (int a = -rp; a <= rp; ++a)
      for (int b = -rp; b <= rp; ++b)
        for (int c = -rp; c <= rp; ++c) {
          const int d[3] = {a, b, c};
          if (!admissible(d, kappa, eta2, wp)) {
            parent_near.insert({a, b, c});
            R = std::max(R, std::max(std::abs(a), std::max(std::abs(b), std::abs(c))));
          }
        }
    const int g = L.grid;
    const int lim = std::min(2 * R + 1, g - 1);
    std::map<std::array<int, 3>, int> op_index;
    std::vector<std::vector<std::array<int, 3>>> alpha_offs(8);
    for (int alpha = 0; alpha < 8; ++alpha) {
      const int al[3] = {alpha & 1, (alpha >> 1) & 1, (alpha >> 2) & 1};
      for (int a = -lim; a <= lim; ++a)
        for (int b = -lim; b <= lim; ++b)
          for (int c = -lim; c <= lim; ++c) {
            const int d[3] = {a, b, c};
            if (!admissible(d, kappa, eta2, L.w)) continue;
            std::array<int, 3> dp;
            for (int i = 0; i < 3; ++i) dp[i] = -floor_div2(al[i] - d[i]);  // ceil((d - alpha)/2)
            if (!parent_near.count(dp)) continue;
            alpha_offs[alpha].push_back({a, b, c});
            op_index.emplace(std::array<int, 3>{a, b, c}, 0);
          }
    }
    int idx = 0;
    for (auto &kv : op_index) {
      kv.second = idx++;
      L.off.insert(L.off.end(), kv.first.begin(), kv.first.end());
      const int d[3] = {kv.first[0], kv.first[1], kv.first[2]};
      L.op_dir.push_back(face_index(plan.l_hf, l, d));
      used[l].insert(L.op_dir.back());
    }
    L.op_base = op_base;
    op_base += idx;
    for (int alpha = 0; alpha < 8; ++alpha)
      for (auto &d : alpha_offs[alpha]) L.alpha_ops[alpha].push_back(op_index[d]);
  }
  plan.n_ops = op_base;
  // direction slots: directions of the level's coupling offsets plus those
  // inherited from the parent level (dir_(l)(c), c used on level l-1)
  for (int l = 1; l <= p; ++l) {
    for (int c : used[l - 1]) {
      const int cc = (l <= plan.l_hf) ? (c >> 2) : 0;
      used[l].insert(cc);
    }
  }
  plan.min_level = p + 1;
  for (int l = p; l >= 0; --l)
    if (!used[l].empty()) plan.min_level = l;
  for (int l = 0; l <= p; ++l) {
    LevelPlan &L = plan.levels[l];
    L.dir_slot.assign(L.ndir_full, -1);
    for (int c : used[l]) {
      L.dir_slot[c] = (int)L.slot_dir.size();
      L.slot_dir.push_back(c);
      double v[3];
      direction_vector(plan.l_hf, l, c, v);
      L.dir_vec.insert(L.dir_vec.end(), v, v + 3);
    }
    // the phase kernels put direction slots on the grid's y dimension
    if (L.slot_dir.size() > 65535)
      throw Error{DFDM_ERR_UNSUPPORTED, "more than 65535 direction slots on one level"};
    for (size_t i = 0; i < L.op_dir.size(); ++i) L.op_slot.push_back(L.dir_slot[L.op_dir[i]]);
    // ops grouped by direction slot; inside a slot by the parity class of d,
    // then by d: consecutive offsets d, d + 2 e_x, ... read source blocks
    // that overlap by three quarters (the M2L reads sources 2 T + alpha - d)
    auto okey = [&](int o) {
      const int *d = &L.off[3 * o];
      const int par = (d[0] & 1) | ((d[1] & 1) << 1) | ((d[2] & 1) << 2);
      return std::make_tuple(L.op_slot[o], par, d[2], d[1], d[0]);
    };
    for (int alpha = 0; alpha < 8; ++alpha) {
      auto &v = L.alpha_ops[alpha];
      std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return okey(a) < okey(b); });
    }
  }
  for (int l = 0; l < p; ++l) {
    LevelPlan &L = plan.levels[l];
    const LevelPlan &C = plan.levels[l + 1];
    for (int c : L.slot_dir) {
      const int cc = (l + 1 <= plan.l_hf) ? (c >> 2) : 0;
      L.child_slot.push_back(C.dir_slot[cc]);
    }
  }
  // nearfield offsets on the leaf level
  plan.near_off.clear();
  {
    const LevelPlan &L = plan.levels[p];
    const int rn = near_radius(kappa, eta2, L.w, L.grid);
    for (int a = -rn; a <= rn; ++a)
      for (int b = -rn; b <= rn; ++b)
        for (int c = -rn; c <= rn; ++c) {
          const int d[3] = {a, b, c};
          if (!admissible(d, kappa, eta2, L.w)) {
            plan.near_off.push_back(a);
            plan.near_off.push_back(b);
            plan.near_off.push_back(c);
          }
        }
  }
}

}  // namespace dfdm
