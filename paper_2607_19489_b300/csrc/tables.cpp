// tables.cpp -- translation operators of the adaptive FMM in box units.
//
// Derivations (g = -1/r, D_gamma(R) = d^gamma g(R); box sizes as in tables.h):
//  M2P  phi(x) = sum_{|a|<=p} (-1)^|a|/a! D_a(x - c) M_a           (Fig. 2, M2P)
//  M2L  L_b    = sum_{|a|+|b|<=p} (-1)^|a|/a! D_{a+b}(c_t - c_s) M_a   (Eq. 3)
//  L2L  L'_b   = sum_{|a|<=p-|b|} d^a/a! L_{a+b}, d = c_child - c_parent (Eq. 4)
//  M2M  M'_a   = sum_{g<=a} C(a,g) d^(a-g) M_g                          (Eq. 2)
// Rescaled to box units these become level independent; the factors below
// (4^-|a-g| 2^-|g| for M2M, 4^-|g-b| 2^-(|b|+1) for L2L, quarter-integer
// target offsets for M2P) are those rescalings for child offsets of +-1/4 of
// the parent box.
#include "tables.h"

#include <cmath>
#include <cstdlib>

namespace fmm {

const int kNbr26[26] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12,
                        14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26};

void MultiIdx::build(int q_) {
  q = q_;
  list.clear();
  lut.assign((q + 1) * (q + 1) * (q + 1), -1);
  for (int n = 0; n <= q; ++n)
    for (int a = n; a >= 0; --a)
      for (int b = n - a; b >= 0; --b) {
        int c = n - a - b;
        lut[(a * (q + 1) + b) * (q + 1) + c] = (int)list.size();
        list.push_back({a, b, c});
      }
}

// Differentiating r^2 d_i f + x_i f = 0 (f = 1/r) with d^gamma (Leibniz) and
// multiplying by r^(2|gamma|+1) gives, for kappa = gamma + e_i,
//   P_kappa = -u_i P_gamma - gamma_i r^2 P_{gamma-e_i}
//             - 2 sum_j gamma_j u_j P_{gamma-e_j+e_i}
//             - r^2 sum_j gamma_j (gamma_j - 1) P_{gamma-2e_j+e_i}.
void inv_r_numerators(int q, const int64_t u[3], std::vector<__int128>& P, const MultiIdx& mi) {
  P.assign(mi.size(), 0);
  __int128 r2 = (__int128)u[0] * u[0] + (__int128)u[1] * u[1] + (__int128)u[2] * u[2];
  P[0] = 1;
  for (int k = 1; k < mi.size(); ++k) {
    const auto& kap = mi.list[k];
    if (kap[0] + kap[1] + kap[2] > q) break;
    int i = kap[0] > 0 ? 0 : (kap[1] > 0 ? 1 : 2);
    std::array<int, 3> g = kap;
    g[i] -= 1;
    auto get = [&](int a, int b, int c) -> __int128 {
      int id = mi.at(a, b, c);
      return id < 0 ? (__int128)0 : P[id];
    };
    __int128 v = -(__int128)u[i] * get(g[0], g[1], g[2]);
    {
      std::array<int, 3> gm = g;
      gm[i] -= 1;
      if (g[i] > 0) v -= (__int128)g[i] * r2 * get(gm[0], gm[1], gm[2]);
    }
    for (int j = 0; j < 3; ++j) {
      if (g[j] == 0) continue;
      std::array<int, 3> t = g;
      t[j] -= 1;
      t[i] += 1;
      v -= (__int128)2 * g[j] * u[j] * get(t[0], t[1], t[2]);
      if (g[j] >= 2) {
        std::array<int, 3> s = g;
        s[j] -= 2;
        s[i] += 1;
        v -= r2 * (__int128)(g[j] * (g[j] - 1)) * get(s[0], s[1], s[2]);
      }
    }
    P[k] = v;
  }
}

namespace {

double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}
double mfact(const std::array<int, 3>& a) { return fact(a[0]) * fact(a[1]) * fact(a[2]); }
double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
int bit(int c, int i) { return (c >> i) & 1; }

// D_gamma(R) = d^gamma(-1/r) at R = u / scale for all |gamma| <= q.
void deriv_g(const int64_t u[3], double scale, int q, const MultiIdx& mi, std::vector<double>& D) {
  std::vector<__int128> P;
  inv_r_numerators(q, u, P, mi);
  long double r2 = (long double)u[0] * u[0] + (long double)u[1] * u[1] + (long double)u[2] * u[2];
  long double r = std::sqrt(r2);
  D.assign(mi.size(), 0.0);
  for (int k = 0; k < mi.size(); ++k) {
    const auto& g = mi.list[k];
    int n = g[0] + g[1] + g[2];
    if (n > q) break;
    // d^g(1/r)(u/s) = s^(n+1) P(u) / |u|^(2n+1)
    long double v = (long double)P[k] * std::pow((long double)scale, n + 1) /
                    (std::pow(r2, (long double)n) * r);
    D[k] = -(double)v;
  }
}

}  // namespace

void Tables::build(int p_, int p_m) {
  p = p_;
  pm = (p_m > 0 && p_m < p) ? p_m : p;
  nc = ncoef(p);
  nc1 = ncoef(p + 1);
  mi.build(p + 1);
  degree.resize(nc);
  for (int a = 0; a < nc; ++a) degree[a] = mi.list[a][0] + mi.list[a][1] + mi.list[a][2];
  const int KQ = 8 * nc, K = 26 * KQ;
  std::vector<double> D;

  // ---- M2P (bottom intermediate field) --------------------------------------
  m2p.assign((size_t)256 * K, 0.0);
  for (int f = 0; f < 8; ++f)
    for (int t = 0; t < 8; ++t)
      for (int qi = 0; qi < 26; ++qi) {
        int q27 = kNbr26[qi];
        int dq[3] = {q27 % 3 - 1, (q27 / 3) % 3 - 1, q27 / 9 - 1};
        for (int s = 0; s < 8; ++s) {
          int rel[3], adj = 1;
          int64_t u[3];
          for (int i = 0; i < 3; ++i) {
            rel[i] = bit(f, i) - 2 * dq[i] - bit(s, i);  // c_F - c_S in level l-1 cells
            if (std::abs(rel[i]) > 1) adj = 0;
            u[i] = 4 * rel[i] + 2 * bit(t, i) - 1;  // 4 (c_t - c_S)
          }
          if (adj) continue;  // S touches F: near field
          deriv_g(u, 4.0, p + 1, mi, D);
          for (int a = 0; a < nc; ++a) {
            if (degree[a] > pm) continue;
            const auto& al = mi.list[a];
            double w = ((degree[a] & 1) ? -1.0 : 1.0) / mfact(al);
            size_t k = (size_t)(qi * 8 + s) * nc + a;
            size_t n0 = (size_t)(f * 8 + t) * 4;
            m2p[(n0 + 0) * K + k] = w * D[mi.at(al[0], al[1], al[2])];
            m2p[(n0 + 1) * K + k] = -w * D[mi.at(al[0] + 1, al[1], al[2])];
            m2p[(n0 + 2) * K + k] = -w * D[mi.at(al[0], al[1] + 1, al[2])];
            m2p[(n0 + 3) * K + k] = -w * D[mi.at(al[0], al[1], al[2] + 1)];
          }
        }
      }

  // ---- M2L (Eq. 3) ------------------------------------------------------------
  m2l.assign((size_t)8 * nc * K, 0.0);
  for (int b = 0; b < 8; ++b)
    for (int qi = 0; qi < 26; ++qi) {
      int q27 = kNbr26[qi];
      int dq[3] = {q27 % 3 - 1, (q27 / 3) % 3 - 1, q27 / 9 - 1};
      for (int s = 0; s < 8; ++s) {
        int64_t u[3];
        int adj = 1;
        for (int i = 0; i < 3; ++i) {
          u[i] = bit(b, i) - 2 * dq[i] - bit(s, i);
          if (std::llabs(u[i]) > 1) adj = 0;
        }
        if (adj) continue;
        deriv_g(u, 1.0, p, mi, D);
        for (int be = 0; be < nc; ++be) {
          const auto& B = mi.list[be];
          for (int a = 0; a < nc; ++a) {
            if (degree[a] + degree[be] > p || degree[a] > pm) continue;
            const auto& al = mi.list[a];
            double w = ((degree[a] & 1) ? -1.0 : 1.0) / mfact(al);
            size_t k = (size_t)(qi * 8 + s) * nc + a;
            size_t n = (size_t)b * nc + be;
            m2l[n * K + k] = w * D[mi.at(al[0] + B[0], al[1] + B[1], al[2] + B[2])];
          }
        }
      }
    }

  // ---- near-field M2P from refined cells at integer offsets ------------------
  nearop.assign((size_t)343 * nc * 4, 0.0);
  for (int z = -3; z <= 3; ++z)
    for (int y = -3; y <= 3; ++y)
      for (int x = -3; x <= 3; ++x) {
        if (std::abs(x) <= 1 && std::abs(y) <= 1 && std::abs(z) <= 1) continue;
        int64_t u[3] = {x, y, z};
        deriv_g(u, 1.0, p + 1, mi, D);
        size_t base = (size_t)((z + 3) * 49 + (y + 3) * 7 + (x + 3)) * nc * 4;
        for (int a = 0; a < nc; ++a) {
          if (degree[a] > pm) continue;
          const auto& al = mi.list[a];
          double w = ((degree[a] & 1) ? -1.0 : 1.0) / mfact(al);
          nearop[base + a * 4 + 0] = w * D[mi.at(al[0], al[1], al[2])];
          nearop[base + a * 4 + 1] = -w * D[mi.at(al[0] + 1, al[1], al[2])];
          nearop[base + a * 4 + 2] = -w * D[mi.at(al[0], al[1] + 1, al[2])];
          nearop[base + a * 4 + 3] = -w * D[mi.at(al[0], al[1], al[2] + 1)];
        }
      }

  // ---- L2P to the 64 grandchild centres of a box --------------------------
  l2p.assign((size_t)64 * nc * 4, 0.0);
  for (int f = 0; f < 8; ++f)
    for (int t = 0; t < 8; ++t) {
      double rho[3];
      for (int i = 0; i < 3; ++i) rho[i] = (bit(f, i) - 0.5) / 2.0 + (bit(t, i) - 0.5) / 4.0;
      size_t base = (size_t)(f * 8 + t) * nc * 4;
      for (int be = 0; be < nc; ++be) {
        const auto& B = mi.list[be];
        double mono = std::pow(rho[0], B[0]) * std::pow(rho[1], B[1]) * std::pow(rho[2], B[2]);
        l2p[base + be * 4 + 0] = mono / mfact(B);
        for (int i = 0; i < 3; ++i) {
          if (B[i] == 0) continue;
          std::array<int, 3> Bm = B;
          Bm[i] -= 1;
          double m2 = std::pow(rho[0], Bm[0]) * std::pow(rho[1], Bm[1]) * std::pow(rho[2], Bm[2]);
          l2p[base + be * 4 + 1 + i] = -m2 / mfact(Bm);  // accel = -grad
        }
      }
    }

  // ---- M2M pair lists -----------------------------------------------------
  m2m_off.assign(1, 0);
  m2m_g.clear();
  m2m_e.clear();
  m2m_c.clear();
  for (int a = 0; a < nc; ++a) {
    const auto& A = mi.list[a];
    for (int g = 0; g < nc; ++g) {
      const auto& Gm = mi.list[g];
      if (Gm[0] > A[0] || Gm[1] > A[1] || Gm[2] > A[2]) continue;
      int e = ((A[0] - Gm[0]) & 1) | (((A[1] - Gm[1]) & 1) << 1) | (((A[2] - Gm[2]) & 1) << 2);
      int dd = degree[a] - degree[g];
      double c = binom(A[0], Gm[0]) * binom(A[1], Gm[1]) * binom(A[2], Gm[2]) *
                 std::ldexp(1.0, -2 * dd - degree[g]);
      m2m_g.push_back(g);
      m2m_e.push_back(e);
      m2m_c.push_back(c);
    }
    m2m_off.push_back((int)m2m_g.size());
  }
  // ---- L2L pair lists, grouped by sign pattern e within each beta ------------
  // l2l_off8[beta*8 + e] .. l2l_off8[beta*8 + e + 1] are the pairs of beta with
  // pattern e, so the device can sum each pattern into its own register.
  l2l_off.assign(1, 0);
  l2l_off8.assign(1, 0);
  l2l_g.clear();
  l2l_e.clear();
  l2l_c.clear();
  for (int be = 0; be < nc; ++be) {
    const auto& B = mi.list[be];
    for (int ee = 0; ee < 8; ++ee) {
      for (int g = 0; g < nc; ++g) {
        const auto& Gm = mi.list[g];
        if (Gm[0] < B[0] || Gm[1] < B[1] || Gm[2] < B[2]) continue;
        std::array<int, 3> al = {Gm[0] - B[0], Gm[1] - B[1], Gm[2] - B[2]};
        int e = (al[0] & 1) | ((al[1] & 1) << 1) | ((al[2] & 1) << 2);
        if (e != ee) continue;
        int da = al[0] + al[1] + al[2];
        double c = std::ldexp(1.0, -2 * da - degree[be] - 1) / mfact(al);
        l2l_g.push_back(g);
        l2l_e.push_back(e);
        l2l_c.push_back(c);
      }
      l2l_off8.push_back((int)l2l_g.size());
    }
    l2l_off.push_back((int)l2l_g.size());
  }
}


void Tables::build_dl2() {
  const int K = 26 * 8 * nc, KP = 26 * 64;
  std::vector<double> D;
  m2p2.assign((size_t)2048 * K, 0.0);
  for (int g = 0; g < 8; ++g)
    for (int qi = 0; qi < 26; ++qi) {
      const int q27 = kNbr26[qi];
      const int dq[3] = {q27 % 3 - 1, (q27 / 3) % 3 - 1, q27 / 9 - 1};
      for (int s = 0; s < 8; ++s) {
        int rel[3], adj = 1;
        for (int i = 0; i < 3; ++i) {
          rel[i] = bit(g, i) - 2 * dq[i] - bit(s, i);  // c_G - c_S in level l-2 cells
          if (std::abs(rel[i]) > 1) adj = 0;
        }
        if (adj) continue;  // S touches G: near field
        for (int f = 0; f < 8; ++f)
          for (int t = 0; t < 8; ++t) {
            int64_t u[3];
            for (int i = 0; i < 3; ++i) u[i] = 8 * rel[i] + 4 * bit(f, i) + 2 * bit(t, i) - 3;  // 8 (c_t - c_S)
            deriv_g(u, 8.0, p + 1, mi, D);
            const size_t n0 = (size_t)((g * 8 + f) * 8 + t) * 4;
            for (int a = 0; a < nc; ++a) {
              if (degree[a] > pm) continue;
              const auto& al = mi.list[a];
              const double w = ((degree[a] & 1) ? -1.0 : 1.0) / mfact(al);
              const size_t k = (size_t)(qi * 8 + s) * nc + a;
              // level l-2 units to level l-1 units: phi x 1/2, accel x 1/4
              m2p2[(n0 + 0) * K + k] = 0.5 * w * D[mi.at(al[0], al[1], al[2])];
              m2p2[(n0 + 1) * K + k] = -0.25 * w * D[mi.at(al[0] + 1, al[1], al[2])];
              m2p2[(n0 + 2) * K + k] = -0.25 * w * D[mi.at(al[0], al[1] + 1, al[2])];
              m2p2[(n0 + 3) * K + k] = -0.25 * w * D[mi.at(al[0], al[1], al[2] + 1)];
            }
          }
      }
    }
  p2pr.assign((size_t)256 * KP, 0.0);
  for (int f = 0; f < 8; ++f)
    for (int qi = 0; qi < 26; ++qi) {
      const int q27 = kNbr26[qi];
      const int dq[3] = {q27 % 3 - 1, (q27 / 3) % 3 - 1, q27 / 9 - 1};
      for (int s = 0; s < 8; ++s) {
        int rel[3], adj = 1;
        for (int i = 0; i < 3; ++i) {
          rel[i] = bit(f, i) - 2 * dq[i] - bit(s, i);  // c_F - c_S in level l-1 cells
          if (std::abs(rel[i]) > 1) adj = 0;
        }
        if (adj) continue;  // S touches F: Delta l = 1's near field
        for (int t = 0; t < 8; ++t)
          for (int kc = 0; kc < 8; ++kc) {
            int64_t u[3];
            for (int i = 0; i < 3; ++i) u[i] = 2 * rel[i] + bit(t, i) - bit(kc, i);  // 2 (c_t - c_child)
            deriv_g(u, 2.0, 1, mi, D);
            const size_t n0 = (size_t)(f * 8 + t) * 4;
            const size_t k = (size_t)(qi * 8 + s) * 8 + kc;
            p2pr[(n0 + 0) * KP + k] = D[mi.at(0, 0, 0)];
            p2pr[(n0 + 1) * KP + k] = -D[mi.at(1, 0, 0)];
            p2pr[(n0 + 2) * KP + k] = -D[mi.at(0, 1, 0)];
            p2pr[(n0 + 3) * KP + k] = -D[mi.at(0, 0, 1)];
          }
      }
    }
}

}  // namespace fmm
