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


// ---- periodic boundaries --------------------------------------------------------
// The lattice tensor by Ewald's split psi = psi_real + psi_recip + pi/a^2 (in the
// g = -1/r convention, psi_real = -sum_n erfc(a|x+n|)/|x+n|, psi_recip =
// -(1/pi) sum_{k != 0} exp(-pi^2 k^2/a^2)/k^2 cos(2 pi k.x)), its Taylor
// coefficients at 0 taken in truncated power-series arithmetic over the three
// coordinates (Taylor-mode differentiation: each term is a function of one
// variable composed with a polynomial in x), then T_gamma = gamma! * coefficient.
namespace {

struct Series {  // truncated power series in (x, y, z), graded order of mi
  const MultiIdx* mi;
  int q;
  std::vector<double> c;
  Series(const MultiIdx& m, int q_) : mi(&m), q(q_), c(m.size(), 0.0) {}
};

Series mul(const Series& a, const Series& b) {
  Series o(*a.mi, a.q);
  const auto& L = a.mi->list;
  for (int i = 0; i < (int)L.size(); ++i) {
    if (a.c[i] == 0.0) continue;
    const int di = L[i][0] + L[i][1] + L[i][2];
    for (int j = 0; j < (int)L.size(); ++j) {
      const int dj = L[j][0] + L[j][1] + L[j][2];
      if (di + dj > a.q) break;  // graded order: degrees only grow
      if (b.c[j] == 0.0) continue;
      o.c[a.mi->at(L[i][0] + L[j][0], L[i][1] + L[j][1], L[i][2] + L[j][2])] += a.c[i] * b.c[j];
    }
  }
  return o;
}

// sum_k f[k] d^k for a series d without constant term (Horner)
Series compose(const std::vector<double>& f, const Series& d) {
  Series o(*d.mi, d.q);
  for (int k = (int)f.size() - 1; k >= 0; --k) {
    o = mul(o, d);
    o.c[0] += f[k];
  }
  return o;
}

// univariate truncated series helpers (coefficients in t)
std::vector<double> umul(const std::vector<double>& a, const std::vector<double>& b) {
  std::vector<double> o(a.size(), 0.0);
  for (size_t i = 0; i < a.size(); ++i)
    for (size_t j = 0; i + j < a.size(); ++j) o[i + j] += a[i] * b[j];
  return o;
}
// (1 + t/s0)^e as a series in t
std::vector<double> upow1(double s0, double e, int q) {
  std::vector<double> o(q + 1, 0.0);
  double c = 1.0;
  for (int k = 0; k <= q; ++k) {
    o[k] = c;
    c *= (e - k) / (k + 1) / s0;
  }
  return o;
}

}  // namespace

std::vector<double> lattice_tensor(int q, const MultiIdx& mi) {
  const double a = 2.0, pi = 3.14159265358979323846, sqpi = std::sqrt(pi);
  Series T(mi, q);
  // real space, n != 0: h(s) = erfc(a sqrt(s)) / sqrt(s) at s = |n + x|^2 = s0 + t,
  // t = 2 n.x + |x|^2 (|n_i| <= 4: beyond, erfc(8) ~ 1e-29)
  const int R = 4;
  for (int nz = -R; nz <= R; ++nz)
    for (int ny = -R; ny <= R; ++ny)
      for (int nx = -R; nx <= R; ++nx) {
        if (!nx && !ny && !nz) continue;
        const double n3[3] = {(double)nx, (double)ny, (double)nz};
        const double s0 = n3[0] * n3[0] + n3[1] * n3[1] + n3[2] * n3[2];
        // y(t) = a sqrt(s0 + t) - y0, a series without constant term
        std::vector<double> y = upow1(s0, 0.5, q);
        const double y0 = a * std::sqrt(s0);
        for (auto& v : y) v *= y0;
        y[0] = 0.0;
        // erfc(y0 + y) = erfc(y0) + sum_k erfc^(k)(y0)/k! y^k, with
        // erfc^(k)(u) = (-1)^k (2/sqrt(pi)) H_{k-1}(u) e^{-u^2} (physicists' Hermite)
        std::vector<double> Hn(q + 1, 0.0), ek(q + 1, 0.0);  // H_n(y0), n < q
        Hn[0] = 1.0;
        if (q >= 2) Hn[1] = 2.0 * y0;
        for (int n = 1; n + 1 < q; ++n) Hn[n + 1] = 2.0 * y0 * Hn[n] - 2.0 * n * Hn[n - 1];
        ek[0] = std::erfc(y0);
        double fk = 1.0;
        for (int k = 1; k <= q; ++k) {
          fk *= k;
          ek[k] = ((k % 2) ? -1.0 : 1.0) * (2.0 / sqpi) * Hn[k - 1] * std::exp(-y0 * y0) / fk;
        }
        std::vector<double> ys(q + 1, 0.0), er(q + 1, 0.0);
        ys[0] = 1.0;  // y^k accumulated
        for (int k = 0; k <= q; ++k) {
          for (int j = 0; j <= q; ++j) er[j] += ek[k] * ys[j];
          ys = umul(ys, y);
        }
        std::vector<double> inv = upow1(s0, -0.5, q);
        for (auto& v : inv) v /= std::sqrt(s0);
        std::vector<double> h = umul(er, inv);  // erfc(a sqrt s)/sqrt s in powers of t
        Series t(mi, q);
        for (int i = 0; i < 3; ++i) {
          int e[3] = {0, 0, 0};
          e[i] = 1;
          if (q >= 1) t.c[mi.at(e[0], e[1], e[2])] += 2.0 * n3[i];  // terms beyond the series' degree drop
          e[i] = 2;
          if (q >= 2) t.c[mi.at(e[0], e[1], e[2])] += 1.0;
        }
        Series f = compose(h, t);
        for (int k = 0; k < mi.size(); ++k) T.c[k] -= f.c[k];
      }
  // n = 0, with g removed: erf(a r)/r = (2a/sqrt(pi)) sum_m (-a^2 s)^m / (m! (2m + 1)), s = |x|^2
  {
    std::vector<double> h(q / 2 + 1, 0.0);
    double fm = 1.0;
    for (int m = 0; m <= q / 2; ++m) {
      if (m) fm *= m;
      h[m] = (2.0 * a / sqpi) * std::pow(-a * a, m) / (fm * (2 * m + 1));
    }
    if (q >= 2) {
      Series s2(mi, q);
      s2.c[mi.at(2, 0, 0)] = s2.c[mi.at(0, 2, 0)] = s2.c[mi.at(0, 0, 2)] = 1.0;
      Series f = compose(h, s2);
      for (int k = 0; k < mi.size(); ++k) T.c[k] += f.c[k];
    } else {
      T.c[0] += h[0];
    }
  }
  // reciprocal space: cos(2 pi k.x) = sum_j (-1)^j (2 pi k.x)^(2j) / (2j)!
  const int kmax = (int)std::ceil(a * std::sqrt(40.0) / pi);
  {
    std::vector<double> cosf(q + 1, 0.0);
    double f = 1.0;
    for (int j = 0; j <= q; ++j) {
      if (j) f *= j;
      if (j % 2 == 0) cosf[j] = (((j / 2) % 2) ? -1.0 : 1.0) / f;
    }
    Series acc(mi, q);
    for (int kz = -kmax; kz <= kmax; ++kz)
      for (int ky = -kmax; ky <= kmax; ++ky)
        for (int kx = -kmax; kx <= kmax; ++kx) {
          if (!kx && !ky && !kz) continue;
          const double k2 = (double)(kx * kx + ky * ky + kz * kz);
          const double w = std::exp(-pi * pi * k2 / (a * a)) / (pi * k2);
          Series th(mi, q);
          if (q >= 1) {
            th.c[mi.at(1, 0, 0)] = 2.0 * pi * kx;
            th.c[mi.at(0, 1, 0)] = 2.0 * pi * ky;
            th.c[mi.at(0, 0, 1)] = 2.0 * pi * kz;
          }
          Series cs = compose(cosf, th);
          for (int k = 0; k < mi.size(); ++k) acc.c[k] += w * cs.c[k];
        }
    for (int k = 0; k < mi.size(); ++k) T.c[k] -= acc.c[k];
  }
  T.c[0] += pi / (a * a);
  // derivatives from Taylor coefficients, then + d^gamma (1/|x|) at the 26 nearest images
  std::vector<double> out(mi.size());
  for (int k = 0; k < mi.size(); ++k) {
    const auto& g = mi.list[k];
    out[k] = T.c[k] * fact(g[0]) * fact(g[1]) * fact(g[2]);
  }
  std::vector<double> D;
  for (int nz = -1; nz <= 1; ++nz)
    for (int ny = -1; ny <= 1; ++ny)
      for (int nx = -1; nx <= 1; ++nx) {
        if (!nx && !ny && !nz) continue;
        const int64_t u[3] = {nx, ny, nz};
        deriv_g(u, 1.0, q, mi, D);  // d^gamma (-1/r)
        for (int k = 0; k < mi.size(); ++k)
          if (mi.list[k][0] + mi.list[k][1] + mi.list[k][2] <= q) out[k] -= D[k];
      }
  return out;
}

void Tables::build_lattice() {
  MultiIdx mq;
  mq.build(p);
  const std::vector<double> T = lattice_tensor(p, mq);
  auto Tat = [&](int a0, int a1, int a2) { return T[mq.at(a0, a1, a2)]; };
  const int K = 8 * nc;
  lattice.assign((size_t)K * K, 0.0);
  const double h1 = 0.5;
  std::vector<double> M0(nc), L0(nc);
  for (int cs = 0; cs < 8; ++cs)
    for (int al = 0; al < nc; ++al) {
      // a unit physical moment alpha of child cs, about its centre, shifted to the root (Eq. 2)
      const auto& A = mi.list[al];
      double d[3];
      for (int i = 0; i < 3; ++i) d[i] = (bit(cs, i) - 0.5) * h1;
      for (int g = 0; g < nc; ++g) {
        const auto& Gm = mi.list[g];
        M0[g] = 0.0;
        if (Gm[0] < A[0] || Gm[1] < A[1] || Gm[2] < A[2]) continue;
        double v = binom(Gm[0], A[0]) * binom(Gm[1], A[1]) * binom(Gm[2], A[2]);
        for (int i = 0; i < 3; ++i) v *= std::pow(d[i], Gm[i] - A[i]);
        M0[g] = v;
      }
      // the lattice M2L at the root (Eq. 3 with D = T, same truncation as M2L)
      for (int be = 0; be < nc; ++be) {
        const auto& B = mi.list[be];
        double v = 0.0;
        for (int g = 0; g < nc; ++g) {
          if (degree[g] + degree[be] > p || degree[g] > pm || M0[g] == 0.0) continue;
          const auto& Gm = mi.list[g];
          v += ((degree[g] & 1) ? -1.0 : 1.0) / mfact(Gm) * Tat(Gm[0] + B[0], Gm[1] + B[1], Gm[2] + B[2]) * M0[g];
        }
        L0[be] = v;
      }
      // L2L (Eq. 4) to each child ct, then to box units of level 1
      for (int ct = 0; ct < 8; ++ct) {
        double r[3];
        for (int i = 0; i < 3; ++i) r[i] = (bit(ct, i) - 0.5) * h1;
        for (int be = 0; be < nc; ++be) {
          const auto& B = mi.list[be];
          double v = 0.0;
          for (int de = 0; de < nc; ++de) {
            if (degree[de] + degree[be] > p) continue;
            const auto& Dl = mi.list[de];
            v += std::pow(r[0], Dl[0]) * std::pow(r[1], Dl[1]) * std::pow(r[2], Dl[2]) / mfact(Dl) *
                 L0[mi.at(Dl[0] + B[0], Dl[1] + B[1], Dl[2] + B[2])];
          }
          lattice[(size_t)(ct * nc + be) * K + cs * nc + al] =
              v * std::pow(h1, degree[be] + 1) * std::pow(h1, degree[al]);
        }
      }
    }
  // Level-1 M2L: all 26 neighbour octs of the one level-1 oct are its own
  // images, so its M2L (box units, the same operator at every level) is a
  // fixed map too; it joins the lattice map and runs in the same FP64 product.
  if (!m2l.empty()) {
    const size_t KM = (size_t)26 * K;
    for (int b = 0; b < 8; ++b)
      for (int be = 0; be < nc; ++be)
        for (int qi = 0; qi < 26; ++qi)
          for (int s2 = 0; s2 < 8; ++s2)
            for (int al = 0; al < nc; ++al)
              lattice[(size_t)(b * nc + be) * K + s2 * nc + al] +=
                  m2l[(size_t)(b * nc + be) * KM + (size_t)(qi * 8 + s2) * nc + al];
  }
}

}  // namespace fmm
