// Host-side FP64 linear algebra for fsgpu: matrix exponential and the adjoint
// of its Frechet derivative, unitarity checks, and the adjacent-pair Givens
// decomposition of an orbital-rotation matrix (§3.2.3).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

#include "fs_internal.h"

namespace fs {

void mat_mul(int n, const zd* A, const zd* B, zd* C) {
  // real arithmetic on the parts (std::complex products carry inf/nan
  // recovery calls that make these small products several times slower)
  std::vector<double> t((size_t)2 * n * n, 0.0);
  const double* a = reinterpret_cast<const double*>(A);
  const double* b = reinterpret_cast<const double*>(B);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const double ar = a[2 * (i * n + k)], ai = a[2 * (i * n + k) + 1];
      if (ar == 0.0 && ai == 0.0) continue;
      double* ti = t.data() + (size_t)2 * i * n;
      const double* bk = b + (size_t)2 * k * n;
      for (int j = 0; j < n; ++j) {
        ti[2 * j] += ar * bk[2 * j] - ai * bk[2 * j + 1];
        ti[2 * j + 1] += ar * bk[2 * j + 1] + ai * bk[2 * j];
      }
    }
  std::copy(t.begin(), t.end(), reinterpret_cast<double*>(C));
}

void mat_adjoint(int n, const zd* A, zd* out) {
  std::vector<zd> t((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) t[j * n + i] = std::conj(A[i * n + j]);
  std::copy(t.begin(), t.end(), out);
}

static double norm1(int n, const zd* A) {
  double m = 0;
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += std::abs(A[i * n + j]);
    m = std::max(m, s);
  }
  return m;
}

// Scaling and squaring with a Taylor series: A / 2^s has 1-norm <= 1/2, and
// the series is summed until a term no longer changes the sum in FP64.
void expm(int n, const zd* A, zd* out) {
  const size_t nn = (size_t)n * n;
  double nrm = norm1(n, A);
  int s = 0;
  if (nrm > 0.5) s = (int)std::ceil(std::log2(nrm / 0.5));
  double scale = std::ldexp(1.0, -s);
  std::vector<zd> B(nn), term(nn), sum(nn, zd(0)), tmp(nn);
  for (size_t k = 0; k < nn; ++k) B[k] = A[k] * scale;
  for (int i = 0; i < n; ++i) {
    sum[i * n + i] = 1.0;
    term[i * n + i] = 1.0;
  }
  for (int k = 1; k <= 40; ++k) {
    mat_mul(n, term.data(), B.data(), tmp.data());
    double tn = 0;
    for (size_t q = 0; q < nn; ++q) {
      term[q] = tmp[q] / (double)k;
      sum[q] += term[q];
      tn = std::max(tn, std::abs(term[q]));
    }
    if (tn < 1e-18) break;
  }
  for (int k = 0; k < s; ++k) mat_mul(n, sum.data(), sum.data(), sum.data());
  std::copy(sum.begin(), sum.end(), out);
}

// For the real inner product <A, B> = Re tr(A^dag B), the adjoint of the
// Frechet derivative of expm at K is the Frechet derivative at K^dag; the
// latter is the upper-right block of expm([[K^dag, H], [0, K^dag]]).
void expm_frechet_adjoint(int n, const zd* K, const zd* H, zd* out) {
  const int m = 2 * n;
  std::vector<zd> B((size_t)m * m, zd(0)), E((size_t)m * m);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      zd kd = std::conj(K[j * n + i]);
      B[i * m + j] = kd;
      B[(n + i) * m + n + j] = kd;
      B[i * m + n + j] = H[i * n + j];
    }
  expm(m, B.data(), E.data());
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) out[i * n + j] = E[i * m + n + j];
}

double unitarity_error(int n, const zd* U) {
  double e = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      zd s = 0;
      for (int k = 0; k < n; ++k) s += std::conj(U[k * n + i]) * U[k * n + j];
      if (i == j) s -= 1.0;
      e = std::max(e, std::abs(s));
    }
  return e;
}

// Column elimination by adjacent Givens rotations from the right: for rows
// r = N-1 .. 1 and columns j = 0 .. r-1, a rotation on columns (j, j+1)
// zeroes A[r][j] and carries the row's weight to column j+1.  With
// A <- A G^dag and G = [[c, s], [-s*, c]] on (j, j+1):
//   new A[r][j] = c a + s* b = 0 for c = |b|/rho, s = -conj(a) b / (|b| rho).
// After all rows A is diagonal: U G_1^dag ... G_M^dag = D, so
// U = D G_M ... G_1 and the operator of G_1 acts first.
RotProgram decompose_adjacent(int n, const zd* U) {
  std::vector<zd> A(U, U + (size_t)n * n);
  RotProgram prog;
  for (int r = n - 1; r >= 1; --r) {
    for (int j = 0; j < r; ++j) {
      zd a = A[r * n + j], b = A[r * n + j + 1];
      if (std::abs(a) == 0.0) continue;  // already zero: identity rotation
      double c;
      zd s;
      if (std::abs(b) == 0.0) {  // swap-like rotation: c = 0, s = -conj(a)/|a|
        c = 0.0;
        s = -std::conj(a) / std::abs(a);
      } else {
        double rho = std::hypot(std::abs(a), std::abs(b));
        c = std::abs(b) / rho;
        s = -std::conj(a) * b / (std::abs(b) * rho);
      }
      // A <- A G^dag on columns (j, j+1): G^dag = [[c, -s], [s*, c]]
      for (int i = 0; i < n; ++i) {
        zd x = A[i * n + j], y = A[i * n + j + 1];
        A[i * n + j] = c * x + std::conj(s) * y;
        A[i * n + j + 1] = -s * x + c * y;
      }
      A[r * n + j] = 0.0;
      prog.g.push_back(Givens{j, c, s});
    }
  }
  prog.phase.resize(n);
  for (int i = 0; i < n; ++i) prog.phase[i] = A[i * n + i];
  return prog;
}

// Greedy grouping of a Givens sequence into window steps: repeatedly take
// the window [a, a+W) that admits the most rotations whose earlier
// neighbours (rotations sharing an orbital and preceding them) are done or
// taken in the same step; the taken rotations keep their relative order, so
// the product of all rotations is unchanged.
std::vector<WinStep> schedule_windows(const RotProgram& rp, int N, int W) {
  const int M = (int)rp.g.size();
  std::vector<char> done(M, 0);
  std::vector<WinStep> steps;
  std::vector<int> taken;
  int nd = 0;
  while (nd < M) {
    WinStep best{0, {}};
    for (int a = 0; a + W <= N; ++a) {
      taken.clear();
      uint64_t blocked = 0;
      for (int k = 0; k < M; ++k) {
        if (done[k]) continue;
        const int p = rp.g[k].p;
        const uint64_t ob = 3ull << p;
        if (ob & blocked) {
          blocked |= ob;
          continue;
        }
        if (p >= a && p + 1 < a + W)
          taken.push_back(k);
        else
          blocked |= ob;
      }
      if (taken.size() > best.givens.size()) best = WinStep{a, taken};
    }
    for (int k : best.givens) done[k] = 1;
    nd += (int)best.givens.size();
    steps.push_back(best);
  }
  return steps;
}

// Top-3 group of a configuration: the occupation of orbitals N-1, N-2, N-3
// read as a 3-bit number (the strings of one group form a contiguous range
// of addresses, since addresses follow the integer order of the masks).
static inline int top3_group(uint32_t mask, int N) {
  return N >= 3 ? (int)((mask >> (N - 3)) & 7u) : 0;
}

// Order of the n items of one class (each reads and writes the 16-byte
// slab cells A[i * ns + k], k < ns, one shared-memory instruction per k)
// for the kernels that deal items to consecutive lanes.  A 16-byte access
// is served eight lanes at a time, and two lanes of those eight that touch
// different cells with equal cell index mod 8 (the same four banks) cost one
// more wavefront.  Greedy: the items are sorted by their pattern of cell
// offsets mod 8 (items with equal patterns and distinct first cells mod 8
// are conflict-free together), then each aligned group of eight is grown
// from the first remaining item by the candidate, among the next kCand,
// that adds the fewest conflicts.  Returns the permutation (new position ->
// old index).
static std::vector<int> bank_order(int n, int ns, const std::vector<int>& A) {
  constexpr int kCand = 128;
  std::vector<int> rem(n);
  std::vector<uint64_t> sig(n);
  for (int i = 0; i < n; ++i) {
    rem[i] = i;
    uint64_t s = 0;
    for (int k = 1; k < ns && k < 22; ++k)
      s |= (uint64_t)((A[(size_t)i * ns + k] - A[(size_t)i * ns]) & 7) << (3 * (k - 1));
    sig[i] = s;
  }
  std::stable_sort(rem.begin(), rem.end(), [&](int u, int v) {
    if (sig[u] != sig[v]) return sig[u] < sig[v];
    return A[(size_t)u * ns] < A[(size_t)v * ns];
  });
  std::vector<int> out;
  out.reserve(n);
  std::vector<int> grp;
  while (!rem.empty()) {
    grp.assign(1, rem.front());
    rem.erase(rem.begin());
    while (grp.size() < 8 && !rem.empty()) {
      int best = 0, bc = 1 << 30;
      const int nc = std::min<int>(kCand, (int)rem.size());
      for (int j = 0; j < nc && bc > 0; ++j) {
        const int i = rem[j];
        int c = 0;
        for (int k = 0; k < ns; ++k) {
          const int cell = A[(size_t)i * ns + k];
          for (int g : grp) {
            const int o = A[(size_t)g * ns + k];
            if (o != cell && ((o ^ cell) & 7) == 0) {
              ++c;
              break;
            }
          }
        }
        if (c < bc) {
          bc = c;
          best = j;
        }
      }
      grp.push_back(rem[best]);
      rem.erase(rem.begin() + best);
    }
    out.insert(out.end(), grp.begin(), grp.end());
  }
  return out;
}

// For the window [a, a+W): every outside configuration O with
// m = n - |O| in 1 .. W-1 is one orbit.  With c_lo = |O below a|, the address
// of O u S (S inside the window) is R_O + F[a][c_lo][S], where R_O sums
// C(o_k, k+1) over O's orbitals with their index k in the full string and F
// sums the same terms over S's orbitals (combinatorial-number-system rank).
void window_tables_host(int N, int n, int W, std::vector<uint32_t>& orbits,
                        std::vector<int>& off, std::vector<uint16_t>& offs,
                        std::vector<uint8_t>& okey) {
  const int npos = N - W + 1;
  orbits.clear();
  okey.clear();
  off.assign(npos + 1, 0);
  offs.assign((size_t)npos * (n + 1) << W, 0);
  auto C = [](int a, int b) -> uint64_t {
    if (b < 0 || b > a) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= b; ++i) r = r * (uint64_t)(a - b + i) / (uint64_t)i;
    return r;
  };
  // Bank-aware order where one CTA holds a whole vector (complex64, psi and
  // g: 16 bytes per string, at most 208 KB); larger spaces run on clusters,
  // whose lists are regrouped by owning CTA, and keep the combinatorial
  // order, under which a warp's strings mostly live on one CTA of the
  // cluster (the bank-aware order made the N = 18 reverse sweeps 19 %
  // slower).
  const bool bank = C(N, n) * 16 <= 208 * 1024;
  for (int a = 0; a < npos; ++a) {
    off[a] = (int)orbits.size();
    std::vector<int> out;
    for (int p = 0; p < N; ++p)
      if (p < a || p >= a + W) out.push_back(p);
    const int no = (int)out.size();
    std::vector<std::vector<uint32_t>> cls(W);
    std::vector<std::vector<uint8_t>> ckey(W);
    for (int m = 1; m < W; ++m) {
      const int ne = n - m;
      if (ne < 0 || ne > no) continue;
      // ne-subsets of the outside orbitals, ascending masks (Gosper's hack)
      uint64_t x = ne == 0 ? 0 : ((1ull << ne) - 1);
      while (true) {
        int clo = 0, k = 0;
        uint64_t ro = 0;
        uint32_t omask = 0;
        for (int i = 0; i < no; ++i)
          if ((x >> i) & 1) {
            int o = out[i];
            omask |= 1u << o;
            if (o < a) {
              ro += C(o, k + 1);
              ++clo;
            } else {
              ro += C(o, k + m + 1);
            }
            ++k;
          }
        cls[m].push_back((uint32_t)ro | ((uint32_t)clo << 16) | ((uint32_t)m << 24));
        ckey[m].push_back((uint8_t)top3_group(omask, N));
        if (ne == 0) break;
        uint64_t c = x & (~x + 1), r = x + c;
        x = (((r ^ x) >> 2) / c) | r;
        if (x >> no) break;
      }
    }
    // Classes in descending order of Givens work per orbit (pairs per
    // rotation C(W-2, m-1), then strings C(W, m)), each padded with empty
    // descriptors (m = 0, skipped by the kernels) to a multiple of 32, so
    // that no warp holds two classes (divergent paths run one after the
    // other) and the per-warp work of a window step is even.
    std::vector<int> order;
    for (int m = 1; m < W; ++m) order.push_back(m);
    std::stable_sort(order.begin(), order.end(), [&](int u, int v) {
      const uint64_t pu = C(W - 2, u - 1), pv = C(W - 2, v - 1);
      return pu != pv ? pu > pv : C(W, u) > C(W, v);
    });
    for (int clo = 0; clo <= n; ++clo)
      for (int S = 0; S < (1 << W); ++S) {
        uint64_t f = 0;
        int j = 0;
        for (int b = 0; b < W; ++b)
          if ((S >> b) & 1) f += C(a + b, clo + (j++) + 1);
        offs[(((size_t)a * (n + 1) + clo) << W) + S] = (uint16_t)std::min<uint64_t>(f, 65535);
      }
    for (int m : order) {
      if (cls[m].empty()) continue;
      // lanes of one shared-memory phase on distinct bank groups
      const int no_m = (int)cls[m].size(), ns = (int)C(W, m);
      std::vector<int> A((size_t)no_m * ns);
      for (int i = 0; i < no_m; ++i) {
        const uint32_t desc = cls[m][i];
        const int RO = desc & 0xFFFF, clo = (desc >> 16) & 0xFF;
        int k = 0;
        for (int S = 0; S < (1 << W); ++S)
          if (__builtin_popcount(S) == m)
            A[(size_t)i * ns + k++] = RO + offs[(((size_t)a * (n + 1) + clo) << W) + S];
      }
      std::vector<int> ord(no_m);
      for (int i = 0; i < no_m; ++i) ord[i] = i;
      if (bank) ord = bank_order(no_m, ns, A);
      for (int i : ord) {
        orbits.push_back(cls[m][i]);
        okey.push_back(ckey[m][i]);
      }
      while ((orbits.size() - off[a]) % 32) {
        orbits.push_back(0u);
        okey.push_back(0);
      }
    }
  }
  off[npos] = (int)orbits.size();
}

}  // namespace fs

namespace fs {

// Subsets of four orbitals covering every unordered orbital pair (greedy:
// repeatedly the subset covering the most uncovered pairs), each pair and
// each diagonal assigned to exactly one subset; and, per subset Q, the
// orbit records of the strings of n electrons: for every configuration O
// outside Q with m = n - |O| in 1..4, the addresses of O u S for the
// C(4, m) subsets S of Q (ascending local masks) and the parities of the
// numbers of O-orbitals in the three gaps of Q.
void tpass_tables_host(int N, int n, std::vector<TPass>& passes,
                       std::vector<TRecord>& recs, std::vector<uint8_t>& rkey) {
  passes.clear();
  recs.clear();
  rkey.clear();
  if (N < 4) return;
  // N = 16: the lines of the affine plane over GF(4), 20 subsets covering
  // every pair exactly once (point (x, y) <-> orbital 4x + y; GF(4) addition
  // is XOR of 2-bit codes, multiplication by the table below).
  // Otherwise: greedy covering, best of several seeded randomized tie-breaks.
  std::vector<std::array<int, 4>> cover;
  if (N == 16) {
    static const int mul[4][4] = {{0, 0, 0, 0}, {0, 1, 2, 3}, {0, 2, 3, 1}, {0, 3, 1, 2}};
    for (int m = 0; m < 4; ++m)
      for (int b = 0; b < 4; ++b) {
        std::array<int, 4> q;
        for (int x = 0; x < 4; ++x) q[x] = 4 * x + (mul[m][x] ^ b);
        std::sort(q.begin(), q.end());
        cover.push_back(q);
      }
    for (int c = 0; c < 4; ++c) cover.push_back({4 * c, 4 * c + 1, 4 * c + 2, 4 * c + 3});
  } else {
    std::vector<std::array<int, 4>> all;
    for (int a = 0; a < N; ++a)
      for (int b = a + 1; b < N; ++b)
        for (int c = b + 1; c < N; ++c)
          for (int d = c + 1; d < N; ++d) all.push_back({a, b, c, d});
    uint64_t rng = 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
      rng ^= rng << 13;
      rng ^= rng >> 7;
      rng ^= rng << 17;
      return rng;
    };
    const int tries = N <= 20 ? 64 : 4;
    for (int t = 0; t < tries; ++t) {
      std::vector<char> cov(N * N, 0);
      std::vector<std::array<int, 4>> cur;
      int left = N * (N - 1) / 2;
      while (left > 0) {
        int best = -1;
        std::vector<int> ties;
        for (size_t i = 0; i < all.size(); ++i) {
          const auto& q = all[i];
          int cnt = 0;
          for (int x = 0; x < 4; ++x)
            for (int y = x + 1; y < 4; ++y) cnt += !cov[q[x] * N + q[y]];
          if (cnt > best) {
            best = cnt;
            ties.clear();
          }
          if (cnt == best) ties.push_back((int)i);
        }
        const auto& q = all[ties[t == 0 ? 0 : next() % ties.size()]];
        for (int x = 0; x < 4; ++x)
          for (int y = x + 1; y < 4; ++y)
            if (!cov[q[x] * N + q[y]]) {
              cov[q[x] * N + q[y]] = 1;
              --left;
            }
        cur.push_back(q);
      }
      if (cover.empty() || cur.size() < cover.size()) cover = cur;
    }
  }
  std::vector<char> pcov(N * N, 0), dcov(N, 0);
  for (const auto& bq : cover) {
    TPass ps{};
    for (int i = 0; i < 4; ++i) ps.q[i] = bq[i];
    ps.keep = 0;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const int p = bq[i], q = bq[j];
        bool take;
        if (i == j) {
          take = !dcov[p];
          dcov[p] = 1;
        } else {
          take = !pcov[std::min(p, q) * N + std::max(p, q)];
        }
        if (take) ps.keep |= 1u << (i * 4 + j);
      }
    for (int i = 0; i < 4; ++i)
      for (int j = i + 1; j < 4; ++j) pcov[bq[i] * N + bq[j]] = 1;
    passes.push_back(ps);
  }
  // diagonals of orbitals not yet assigned
  for (int p = 0; p < N; ++p)
    if (!dcov[p]) {
      for (auto& ps : passes)
        for (int i = 0; i < 4; ++i)
          if (ps.q[i] == p && !dcov[p]) {
            ps.keep |= 1u << (i * 5);
            dcov[p] = 1;
          }
    }
  auto C = [](int a, int b) -> uint64_t {
    if (b < 0 || b > a) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= b; ++i) r = r * (uint64_t)(a - b + i) / (uint64_t)i;
    return r;
  };
  auto rank = [&](uint32_t mask) {
    uint64_t r = 0;
    int k = 0;
    for (int o = 0; o < N; ++o)
      if ((mask >> o) & 1u) r += C(o, ++k);
    return r;
  };
  for (auto& ps : passes) {
    ps.rec0 = (int)recs.size();
    uint32_t qmask = 0;
    for (int i = 0; i < 4; ++i) qmask |= 1u << ps.q[i];
    std::vector<int> out;
    for (int p = 0; p < N; ++p)
      if (!((qmask >> p) & 1u)) out.push_back(p);
    const int no = (int)out.size();
    std::vector<TRecord> rcls[5];
    std::vector<uint8_t> rck[5];
    for (int m = 1; m <= 4; ++m) {
      const int ne = n - m;
      if (ne < 0 || ne > no) continue;
      uint64_t x = ne == 0 ? 0 : ((1ull << ne) - 1);
      while (true) {
        uint32_t omask = 0;
        for (int i = 0; i < no; ++i)
          if ((x >> i) & 1) omask |= 1u << out[i];
        TRecord r{};
        int k = 0;
        for (int s = 0; s < 16; ++s) {
          if (__builtin_popcount(s) != m) continue;
          uint32_t full = omask;
          for (int i = 0; i < 4; ++i)
            if ((s >> i) & 1) full |= 1u << ps.q[i];
          r.addr[k++] = (uint16_t)rank(full);
        }
        r.m = (uint8_t)m;
        uint8_t g = 0, acc = 0;
        for (int j = 0; j < 3; ++j) {
          uint32_t gap = ((1u << ps.q[j + 1]) - 1u) & ~((2u << ps.q[j]) - 1u);
          acc ^= (uint8_t)(__builtin_popcount(omask & gap) & 1);
          g |= (uint8_t)(acc << (j + 1));  // bit j+1: parity of O before q_{j+1}
        }
        r.gbits = g;
        // omega(S) for each local subset S in the record's order
        r.flips = 0;
        for (int s = 0, kk = 0; s < 16; ++s) {
          if (__builtin_popcount(s) != m) continue;
          int f = 0;
          for (int j = 1; j < 4; ++j)
            if ((s >> j) & 1) f ^= (g >> j) & 1;
          r.flips |= (uint16_t)(f << kk++);
        }
        rcls[m].push_back(r);
        rck[m].push_back((uint8_t)top3_group(omask, N));
        if (ne == 0) break;
        uint64_t c = x & (~x + 1), rr = x + c;
        x = (((rr ^ x) >> 2) / c) | rr;
        if (x >> no) break;
      }
    }
    // Classes in descending order of work per record (terms of the local
    // pairs: 36, 24, 16, 4 for m = 2, 3, 1, 4), each padded with empty
    // records (m = 0, skipped by the kernels) to a multiple of 32.
    for (int m : {2, 3, 1, 4}) {
      if (rcls[m].empty()) continue;
      // lanes of one shared-memory phase on distinct bank groups
      const int nr = (int)rcls[m].size(), ns = (int)C(4, m);
      std::vector<int> A((size_t)nr * ns);
      for (int i = 0; i < nr; ++i)
        for (int k = 0; k < ns; ++k) A[(size_t)i * ns + k] = rcls[m][i].addr[k];
      std::vector<int> ord(nr);
      for (int i = 0; i < nr; ++i) ord[i] = i;
      if (C(N, n) * 16 <= 208 * 1024) ord = bank_order(nr, ns, A);  // as for the windows
      for (int i : ord) {
        recs.push_back(rcls[m][i]);
        rkey.push_back(rck[m][i]);
      }
      while ((recs.size() - ps.rec0) % 32) {
        recs.push_back(TRecord{});
        rkey.push_back(0);
      }
    }
    ps.rec1 = (int)recs.size();
  }
}

// Regrouping of an item list for clusters of 2^b CTAs: within each segment
// [seg[i], seg[i + 1]) the items are stably reordered by their top-b group
// key >> (3 - b) (keeping the class order inside a group, each class of a
// group padded to a multiple of 32 again);
// gofs[i * 9 + r] is the
// start of group r of segment i (r = 0 .. 2^b, the last entry the segment
// end).
static bool is_padding(uint32_t orbit) { return (orbit >> 24) == 0; }
static bool is_padding(const TRecord& r) { return r.m == 0; }
static int item_class(uint32_t orbit) { return (int)(orbit >> 24); }
static int item_class(const TRecord& r) { return r.m; }

template <typename T>
static void regroup(const std::vector<T>& items, const std::vector<uint8_t>& key,
                    const std::vector<int>& seg, int b, std::vector<T>& out,
                    std::vector<int>& gofs) {
  const int ns = (int)seg.size() - 1, G = 1 << b;
  out.clear();
  out.reserve(items.size());
  gofs.assign((size_t)std::max(ns, 0) * 9, 0);
  for (int i = 0; i < ns; ++i) {
    for (int r = 0; r < G; ++r) {
      const size_t g0 = out.size();
      gofs[(size_t)i * 9 + r] = (int)g0;
      int cur = -1;
      for (int k = seg[i]; k < seg[i + 1]; ++k) {
        if ((key[k] >> (3 - b)) != r || is_padding(items[k])) continue;
        if (item_class(items[k]) != cur) {  // a new class starts on a warp
          while ((out.size() - g0) % 32) out.push_back(T{});
          cur = item_class(items[k]);
        }
        out.push_back(items[k]);
      }
      while ((out.size() - g0) % 32) out.push_back(T{});
    }
    for (int r = G; r <= 8; ++r) gofs[(size_t)i * 9 + r] = (int)out.size();
  }
}

void window_groups_host(const std::vector<uint32_t>& orbits, const std::vector<int>& off,
                        const std::vector<uint8_t>& okey, int b, std::vector<uint32_t>& gorb,
                        std::vector<int>& goff) {
  regroup(orbits, okey, off, b, gorb, goff);
}

void tpass_groups_host(const std::vector<TPass>& passes, const std::vector<TRecord>& recs,
                       const std::vector<uint8_t>& rkey, int b, std::vector<TRecord>& grec,
                       std::vector<int>& goff) {
  std::vector<int> seg;
  for (const auto& p : passes) seg.push_back(p.rec0);
  seg.push_back(passes.empty() ? 0 : passes.back().rec1);
  regroup(recs, rkey, seg, b, grec, goff);
}

}  // namespace fs
