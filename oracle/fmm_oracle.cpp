// fmm_oracle.cpp -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, FP64 CPU implementation of the adaptive FMM Poisson solver of
// Lee & Teyssier, "A Scalable FMM Poisson Solver for the RAMSES code: II. AMR
// and Adaptive Time Stepping" (arXiv 2607.19489).  It exists to check the CUDA
// library against the paper.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark may load it; the product path never does.  It
// shares no code, header, table or helper with the CUDA library.
//
// It follows the paper literally:
//   * one sparse FMM tree T_j per AMR level j, holding multipoles of level-j
//     cells only, on FMM grids 1..j-1                       (Sec. 3.1)
//   * Upward = P2M (Eq. 1) + M2M (Eq. 2) about box centres  (Alg. 2)
//   * merged tree = sum of trees j >= l+1, rebuilt per target level (Alg. 1)
//   * MultipoleToLocal: L2L (Eq. 4) + M2L (Eq. 3) / P2L over the 6^3-3^3
//     interaction list, one contribution per tree       (Sec. 2, Alg. 3)
//   * PotentialEvaluation: far (L2P), intermediate (P2P / M2P from T_l and the
//     merged tree), near and nearest fields             (Sec. 3.2, Fig. 2, Alg. 4)
// It loops target by target and source by source; no blocking, no GEMMs.
//
// Conventions (readings of the paper where it is silent):
//   * box [0,1)^3, level-l cell size h = 2^-l, cells are point masses at their
//     centres (footnote on P2M in Sec. 2);
//   * g(R) = -1/|R|, phi = G * sum g * m, accel = -grad phi;
//   * multipole order = local order = p, M2L truncated at |alpha|+|beta| <= p
//     (Eq. 3), M2P at |alpha| <= p;
//   * M2L at box levels 2..l-2, L2P from the level l-2 box, M2P at level l-1;
//   * self-interaction excluded; targets are leaf cells only; isolated
//     boundaries (nothing outside the unit box).
// Two options beside the paper's defaults:
//   * multipole order p_m <= p: Eq. 3 sums n <= p - m over the multipoles that
//     exist; the paper's quadrupoles with p = 3 are p_m = 2.  M2L keeps
//     |alpha| <= p_m and |alpha| + |beta| <= p, M2P keeps |alpha| <= p_m;
//   * bottom mode 1: the sources of the interaction list of the target's parent
//     box F (level l-1) reach the target through F's local expansion (M2L / P2L
//     into F, which also receives L2L from its parent, then L2P), instead of
//     M2P / P2P to the target (Fig. 2, Alg. 4).  The downward pass then runs to
//     box level l-1 and the far field is the L2P of F.
//   * multipole drifting (Sec. 4 names it as future work, after SWIFT): in a
//     solve from level lo, every box of a stale tree T_j (j < lo) is moved by
//     the centre-of-mass velocity of T_j's cells inside it times dt[j], the time
//     since level j was last set: its moments about the box centre c become the
//     moments of the moved mass, i.e. the moments about c - d (the shift of
//     Eq. 2 with displacement d).  Cells used as point masses (P2P, P2L) stay
//     at their centres.
//
// A third option, for a single complete level only:
//   * Delta l = 2 (the footnote of Sec. 2: Paper I's generalisation, tested
//     there on unigrids; the paper keeps Delta l = 1 for AMR and ATS): the
//     finest FMM box holds the 4^3 cells two levels up instead of an oct's
//     2^3.  The downward pass stops at box level l-3 (far field = L2P of the
//     level l-3 ancestor), the bottom intermediate field is the M2P from the
//     interaction list of the target's level l-2 ancestor G, and the near field
//     is the direct sum over the cells of G's 3^3 neighbours (12^3 = 1728
//     cells less the target).
//
// Periodic boundaries (an extension: Sec. 6 names periodic domains as the next
// step for cosmology without fixing a method).  The unit box tiles space, every
// cell has images at all integer offsets n, and a uniform background of the
// opposite total mass makes the problem solvable (lap phi = 4 pi G (rho -
// mean rho)).  The pair potential is Ewald's lattice sum, written in this
// solver's sign convention g = -1/r (box volume 1, splitting parameter a):
//   psi(r) = -[ sum_n erfc(a|r+n|)/|r+n|
//               + (1/pi) sum_{k != 0} exp(-pi^2 k^2 / a^2) / k^2 cos(2 pi k.r) - pi/a^2 ]
// which does not depend on a and has zero mean over the box.  A cell's own
// images act on it (psi minus its 1/r singularity).  The FMM reading: every
// neighbour and interaction list wraps around the box at every level (the
// geometry is that of the image, the content that of the wrapped box); the
// root's 3^3 images reach the targets through the lists of levels 1 and
// below, with M2L now also at box level 1; every farther image, and the
// background, reaches the root's local expansion through the lattice tensor
// T_gamma = d^gamma psi_far(0), psi_far = psi minus the 27 nearest images of
// g (Eq. 3 with D = T and the root multipole as the source), which L2L hands
// down to level 1.  Periodic solves need lmin >= 3.
//
// Parity status: pinned by the tests in tests/test_oracle_*.py against the
// O(N^2) direct sum (exact agreement where the FMM has no far field, error
// falling with p elsewhere), closed forms of the derivatives of 1/r, the M2M
// and L2L exactness identities, linearity, mirror symmetry and the exact
// antisymmetry of nearest-field pairs.

#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <set>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using I3 = std::array<int, 3>;
using Vec = std::vector<double>;

enum {
  ORC_OK = 0,
  ORC_ERR_ARG = -1,
  ORC_ERR_NOT_GRADED = -2,
  ORC_ERR_DUPLICATE = -3,
  ORC_ERR_OUT_OF_BOX = -4,
  ORC_ERR_INCOMPLETE = -10,
};

// ---------------------------------------------------------------------------
// Multi-indices alpha = (a,b,c), |alpha| <= q, graded order: degree n = 0..q,
// within a degree a descending, then b descending.
struct MultiIndex {
  int q = -1;
  std::vector<I3> list;
  std::map<I3, int> index;
  void build(int q_) {
    q = q_;
    list.clear();
    index.clear();
    for (int n = 0; n <= q; ++n)
      for (int a = n; a >= 0; --a)
        for (int b = n - a; b >= 0; --b) {
          I3 m{a, b, n - a - b};
          index[m] = (int)list.size();
          list.push_back(m);
        }
  }
  int at(int a, int b, int c) const { return index.at(I3{a, b, c}); }
  int size() const { return (int)list.size(); }
};

double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}
double mfact(const I3& a) { return factorial(a[0]) * factorial(a[1]) * factorial(a[2]); }
int deg(const I3& a) { return a[0] + a[1] + a[2]; }
double ipow(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}
double mpow(const double* x, const I3& a) {
  return ipow(x[0], a[0]) * ipow(x[1], a[1]) * ipow(x[2], a[2]);
}
double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// ---------------------------------------------------------------------------
// Derivatives of 1/r by symbolic differentiation.  d^gamma (1/r) = P_gamma(x) /
// r^(2|gamma|+1) with P_gamma an integer polynomial; differentiating the
// quotient once more in direction i gives
//     P_{gamma+e_i} = r^2 * dP_gamma/dx_i - (2|gamma|+1) * x_i * P_gamma.
// The Green's function of Sec. 2 (Eq. 3) is g = -1/r, so d^gamma g = -P/r^...
using Poly = std::map<I3, long long>;

struct Derivs {
  int q = -1;
  MultiIndex mi;
  std::vector<Poly> P;  // indexed like mi.list
  void build(int q_) {
    if (q_ <= q) return;
    q = q_;
    mi.build(q);
    P.assign(mi.size(), Poly());
    P[0][I3{0, 0, 0}] = 1;
    for (int k = 1; k < mi.size(); ++k) {
      I3 g = mi.list[k];
      int i = (g[0] > 0) ? 0 : (g[1] > 0 ? 1 : 2);
      I3 gp = g;
      gp[i] -= 1;
      const Poly& src = P[mi.at(gp[0], gp[1], gp[2])];
      int n = deg(gp);
      Poly out;
      for (const auto& kv : src) {
        I3 e = kv.first;
        long long c = kv.second;
        if (e[i] > 0) {  // r^2 * dP/dx_i
          I3 d = e;
          long long cd = c * e[i];
          d[i] -= 1;
          for (int j = 0; j < 3; ++j) {
            I3 t = d;
            t[j] += 2;
            out[t] += cd;
          }
        }
        I3 t = e;  // -(2n+1) x_i P
        t[i] += 1;
        out[t] -= (long long)(2 * n + 1) * c;
      }
      Poly clean;
      for (const auto& kv : out)
        if (kv.second != 0) clean[kv.first] = kv.second;
      P[k] = clean;
    }
  }
  // d^gamma(1/r) at R for all |gamma| <= q (mi order)
  void inv_r(const double* R, double* out) const {
    double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    double r = std::sqrt(r2);
    for (int k = 0; k < mi.size(); ++k) {
      double s = 0.0;
      for (const auto& kv : P[k]) s += (double)kv.second * mpow(R, kv.first);
      s /= ipow(r, 2 * deg(mi.list[k]) + 1);
      out[k] = s;
    }
  }
  long long numerator(int k, const long long* u) const {
    long long s = 0;
    for (const auto& kv : P[k]) {
      long long m = kv.second;
      for (int j = 0; j < 3; ++j)
        for (int e = 0; e < kv.first[j]; ++e) m *= u[j];
      s += m;
    }
    return s;
  }
};

Derivs g_der;
std::mutex g_der_mu;
void ensure_derivs(int q) {
  std::lock_guard<std::mutex> lk(g_der_mu);
  g_der.build(q);
}

// D_gamma = d^gamma g(R), g = -1/r, for |gamma| <= q, memoised per thread by R.
struct DCache {
  int q;
  std::map<std::array<double, 3>, Vec> memo;
  explicit DCache(int q_) : q(q_) {}
  const Vec& get(const double* R) {
    std::array<double, 3> key{R[0], R[1], R[2]};
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    int n = (q + 1) * (q + 2) * (q + 3) / 6;
    Vec d(g_der.mi.size());
    g_der.inv_r(R, d.data());  // g_der built to >= q; its first n entries are |gamma|<=q
    d.resize(n);
    for (auto& v : d) v = -v;
    return memo.emplace(key, std::move(d)).first->second;
  }
};

// ---------------------------------------------------------------------------
// Expansion operators, each written from its equation.  Coordinates physical.
struct Ops {
  int p;
  int pm;          // multipole order of M2L and M2P (<= p)
  MultiIndex mi;   // |alpha| <= p
  MultiIndex mi1;  // |alpha| <= p+1 (matches g_der.mi prefix)
  explicit Ops(int p_, int pm_ = 0) : p(p_), pm(pm_ > 0 && pm_ < p_ ? pm_ : p_) {
    mi.build(p);
    mi1.build(p + 1);
  }
  int n() const { return mi.size(); }

  // Eq. (1): M_alpha += m (x - c)^alpha
  void p2m(double m, const double* x, const double* c, Vec& M) const {
    double d[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
    for (int k = 0; k < n(); ++k) M[k] += m * mpow(d, mi.list[k]);
  }
  // Eq. (2): moments about c_child shifted to c_parent:
  // M'_alpha = sum_{gamma<=alpha} C(alpha,gamma) (c_child - c_parent)^(alpha-gamma) M_gamma
  void m2m(const Vec& Mc, const double* cc, const double* cp, Vec& Mp) const {
    double d[3] = {cc[0] - cp[0], cc[1] - cp[1], cc[2] - cp[2]};
    for (int k = 0; k < n(); ++k) {
      const I3& a = mi.list[k];
      double s = 0.0;
      for (int g0 = 0; g0 <= a[0]; ++g0)
        for (int g1 = 0; g1 <= a[1]; ++g1)
          for (int g2 = 0; g2 <= a[2]; ++g2) {
            I3 rest{a[0] - g0, a[1] - g1, a[2] - g2};
            double c = binom(a[0], g0) * binom(a[1], g1) * binom(a[2], g2);
            s += c * mpow(d, rest) * Mc[mi.at(g0, g1, g2)];
          }
      Mp[k] += s;
    }
  }
  // Eq. (3): L_beta += sum_{|alpha|<=p-|beta|, |alpha|<=pm} (-1)^|alpha|/alpha! D_{alpha+beta}(c_t - c_s) M_alpha
  void m2l(const Vec& M, const Vec& D, Vec& L) const {
    for (int kb = 0; kb < n(); ++kb) {
      const I3& b = mi.list[kb];
      double s = 0.0;
      for (int ka = 0; ka < n(); ++ka) {
        const I3& a = mi.list[ka];
        if (deg(a) + deg(b) > p || deg(a) > pm) continue;
        double sg = (deg(a) % 2) ? -1.0 : 1.0;
        s += sg / mfact(a) * D[mi1.at(a[0] + b[0], a[1] + b[1], a[2] + b[2])] * M[ka];
      }
      L[kb] += s;
    }
  }
  // P2L: a point mass m at the source centre: L_beta += m D_beta
  void p2l(double m, const Vec& D, Vec& L) const {
    for (int kb = 0; kb < n(); ++kb) L[kb] += m * D[kb];
  }
  // Eq. (4): L'_beta = sum_{|alpha|<=p-|beta|} a^alpha/alpha! L_{alpha+beta}, a = c_child - c_parent
  void l2l(const Vec& Lp, const double* cp, const double* cc, Vec& Lc) const {
    double a[3] = {cc[0] - cp[0], cc[1] - cp[1], cc[2] - cp[2]};
    for (int kb = 0; kb < n(); ++kb) {
      const I3& b = mi.list[kb];
      double s = 0.0;
      for (int ka = 0; ka < n(); ++ka) {
        const I3& al = mi.list[ka];
        if (deg(al) + deg(b) > p) continue;
        s += mpow(a, al) / mfact(al) * Lp[mi.at(al[0] + b[0], al[1] + b[1], al[2] + b[2])];
      }
      Lc[kb] += s;
    }
  }
  // Local expansion evaluated at x: phi = sum L_beta r^beta/beta!, and its exact gradient.
  void l2p(const Vec& L, const double* c, const double* x, double* phi, double* grad) const {
    double r[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
    for (int k = 0; k < n(); ++k) {
      const I3& b = mi.list[k];
      double f = mfact(b);
      *phi += L[k] * mpow(r, b) / f;
      for (int i = 0; i < 3; ++i) {
        if (b[i] == 0) continue;
        I3 bm = b;
        bm[i] -= 1;
        grad[i] += L[k] * b[i] * mpow(r, bm) / f;
      }
    }
  }
  // M2P: phi = sum_{|alpha|<=pm} (-1)^|alpha|/alpha! D_alpha(x - c) M_alpha;
  // d phi/dx_i uses D_{alpha+e_i}.  D must hold |gamma| <= p+1.
  void m2p(const Vec& M, const Vec& D, double* phi, double* grad) const {
    for (int k = 0; k < n(); ++k) {
      const I3& a = mi.list[k];
      if (deg(a) > pm) continue;
      double w = ((deg(a) % 2) ? -1.0 : 1.0) / mfact(a) * M[k];
      *phi += w * D[mi1.at(a[0], a[1], a[2])];
      grad[0] += w * D[mi1.at(a[0] + 1, a[1], a[2])];
      grad[1] += w * D[mi1.at(a[0], a[1] + 1, a[2])];
      grad[2] += w * D[mi1.at(a[0], a[1], a[2] + 1)];
    }
  }
};

// P2P: potential g(x-y) m = -m/|x-y| and its gradient m (x-y)/|x-y|^3.
inline void p2p(double m, const double* y, const double* x, double* phi, double* grad) {
  double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double r = std::sqrt(r2);
  double ir = 1.0 / r;
  double ir3 = ir / r2;
  *phi -= m * ir;
  grad[0] += m * d[0] * ir3;
  grad[1] += m * d[1] * ir3;
  grad[2] += m * d[2] * ir3;
}

// ---------------------------------------------------------------------------
// Periodic boundaries: Ewald's pair potential psi (see the header) and the
// lattice tensor of the root.
constexpr double kPi = 3.14159265358979323846;

// psi(r) and grad psi(r) for r in (-1, 1)^3, r != 0.  With a >= 6 every image
// beyond the 27 around r adds less than erfc(a) (< 2e-17), and the reciprocal
// sum stops where exp(-pi^2 k^2 / a^2) < exp(-40).
struct Ewald {
  double a;
  int kmax;
  std::vector<std::array<double, 4>> kv;  // (kx, ky, kz, weight (1/pi) exp(-pi^2 k^2/a^2)/k^2)
  explicit Ewald(double a_) : a(a_) {
    kmax = (int)std::ceil(a * std::sqrt(40.0) / kPi);
    for (int z = -kmax; z <= kmax; ++z)
      for (int y = -kmax; y <= kmax; ++y)
        for (int x = -kmax; x <= kmax; ++x) {
          if (!x && !y && !z) continue;
          double k2 = (double)(x * x + y * y + z * z);
          double w = std::exp(-kPi * kPi * k2 / (a * a)) / (kPi * k2);
          if (w < 1e-300) continue;
          kv.push_back({(double)x, (double)y, (double)z, w});
        }
  }
  // erfc(a rho)/rho and its derivative factor: grad = -x (erfc(a rho) + 2 a rho e^{-a^2 rho^2}/sqrt(pi)) / rho^3
  void real(const double* x, double* v, double* g) const {
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double r = std::sqrt(r2);
    double e = std::erfc(a * r);
    *v += e / r;
    double f = -(e + 2.0 * a * r * std::exp(-a * a * r2) / std::sqrt(kPi)) / (r2 * r);
    for (int i = 0; i < 3; ++i) g[i] += f * x[i];
  }
  // psi and grad psi at r (r not a lattice point)
  void pair(const double* r, double* psi, double* grad) const {
    double v = 0.0, g[3] = {0.0, 0.0, 0.0};
    for (int nz = -1; nz <= 1; ++nz)
      for (int ny = -1; ny <= 1; ++ny)
        for (int nx = -1; nx <= 1; ++nx) {
          double x[3] = {r[0] + nx, r[1] + ny, r[2] + nz};
          real(x, &v, g);
        }
    for (const auto& k : kv) {
      double ph = 2.0 * kPi * (k[0] * r[0] + k[1] * r[1] + k[2] * r[2]);
      v += k[3] * std::cos(ph);
      double s = -k[3] * 2.0 * kPi * std::sin(ph);
      for (int i = 0; i < 3; ++i) g[i] += s * k[i];
    }
    v -= kPi / (a * a);
    *psi = -v;
    for (int i = 0; i < 3; ++i) grad[i] = -g[i];
  }
  // lim_{r -> 0} psi(r) + 1/r: what a cell's own images (and the background) add
  double self() const {
    double v = 0.0, g[3];
    for (int nz = -1; nz <= 1; ++nz)
      for (int ny = -1; ny <= 1; ++ny)
        for (int nx = -1; nx <= 1; ++nx) {
          if (!nx && !ny && !nz) continue;
          double x[3] = {(double)nx, (double)ny, (double)nz};
          real(x, &v, g);
        }
    for (const auto& k : kv) v += k[3];
    v += -kPi / (a * a) - 2.0 * a / std::sqrt(kPi);
    return -v;
  }
};

// Lattice tensor T_gamma = d^gamma psi_far(0), |gamma| <= q, where psi_far is
// psi minus g over the 27 images n in {-1,0,1}^3.  By the Ewald split:
//   T = -sum_{n != 0} d^gamma [erfc(a|x|)/|x|](n) + d^gamma [erf(a r)/r](0)
//       - (1/pi) sum_k e^{-pi^2 k^2/a^2}/k^2 d^gamma cos(2 pi k.x)(0) + pi/a^2 [gamma = 0]
//       + sum_{n in 27, n != 0} d^gamma (1/|x|)(n).
// The real-space derivatives of the radial f(rho) = erfc(a rho)/rho use
// d_i f_k = x_i f_{k+1} with f_k = (rho^-1 d/drho)^k f = (-1)^k B_k and
// B_k = ((2k - 1) B_{k-1} + (2a^2)^k e^{-a^2 rho^2} / (a sqrt(pi))) / rho^2, so
// d^gamma f = sum_k c_{gamma,k}(x) f_k with polynomials c built by the product rule.
struct RadialPoly {  // sum over (x^e, k) of coefficient * x^e * f_k
  std::map<std::array<int, 4>, double> t;
};

Vec lattice_tensor(int q, double a) {
  MultiIndex mi;
  mi.build(q);
  const int nq = mi.size();
  // product-rule polynomials for every gamma, built from gamma - e_i
  std::vector<RadialPoly> C(nq);
  C[0].t[{0, 0, 0, 0}] = 1.0;
  for (int k = 1; k < nq; ++k) {
    I3 gmm = mi.list[k];
    int i = (gmm[0] > 0) ? 0 : (gmm[1] > 0 ? 1 : 2);
    I3 gp = gmm;
    gp[i] -= 1;
    const RadialPoly& src = C[mi.at(gp[0], gp[1], gp[2])];
    RadialPoly out;
    for (const auto& kv : src.t) {
      std::array<int, 4> e = kv.first;
      if (e[i] > 0) {  // derivative of the monomial
        std::array<int, 4> d = e;
        d[i] -= 1;
        out.t[d] += kv.second * e[i];
      }
      std::array<int, 4> u = e;  // x_i f_{k+1}
      u[i] += 1;
      u[3] += 1;
      out.t[u] += kv.second;
    }
    C[k] = out;
  }
  Vec T(nq, 0.0);
  // real space, n != 0, |n_i| <= 5 (erfc(2a) and beyond are below 1e-40 for a = 2)
  const int R = 5;
  for (int nz = -R; nz <= R; ++nz)
    for (int ny = -R; ny <= R; ++ny)
      for (int nx = -R; nx <= R; ++nx) {
        if (!nx && !ny && !nz) continue;
        double x[3] = {(double)nx, (double)ny, (double)nz};
        double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        double r = std::sqrt(r2);
        std::vector<double> f(q + 1);
        double B = std::erfc(a * r) / r;
        f[0] = B;
        for (int k = 1; k <= q; ++k) {
          B = ((2 * k - 1) * B + std::pow(2.0 * a * a, k) * std::exp(-a * a * r2) / (a * std::sqrt(kPi))) / r2;
          f[k] = (k % 2) ? -B : B;
        }
        for (int k = 0; k < nq; ++k) {
          double s = 0.0;
          for (const auto& kv : C[k].t) {
            const auto& e = kv.first;
            s += kv.second * mpow(x, I3{e[0], e[1], e[2]}) * f[e[3]];
          }
          T[k] -= s;
        }
      }
  // n = 0: erf(a r)/r = (2a/sqrt(pi)) sum_m (-1)^m a^{2m} r^{2m} / (m! (2m+1));
  // d^gamma r^{2m} at 0 is nonzero only for gamma = 2 (a, b, c), a + b + c = m:
  // m!/(a! b! c!) (2a)! (2b)! (2c)!
  for (int k = 0; k < nq; ++k) {
    const I3& g = mi.list[k];
    if ((g[0] | g[1] | g[2]) & 1) continue;
    int m = deg(g) / 2;
    double coef = (2.0 * a / std::sqrt(kPi)) * ((m % 2) ? -1.0 : 1.0) * std::pow(a, 2 * m) /
                  (factorial(m) * (2 * m + 1));
    double d = factorial(m) / (factorial(g[0] / 2) * factorial(g[1] / 2) * factorial(g[2] / 2)) *
               factorial(g[0]) * factorial(g[1]) * factorial(g[2]);
    T[k] += coef * d;
  }
  // reciprocal space: d^gamma cos(2 pi k.x) at 0 = (2 pi)^|gamma| k^gamma (-1)^{|gamma|/2}, |gamma| even
  Ewald ew(a);
  for (int k = 0; k < nq; ++k) {
    const I3& g = mi.list[k];
    int n = deg(g);
    if (n % 2) continue;
    double sgn = ((n / 2) % 2) ? -1.0 : 1.0;
    double s = 0.0;
    for (const auto& kk : ew.kv) {
      double kvv[3] = {kk[0], kk[1], kk[2]};
      s += kk[3] * mpow(kvv, g);
    }
    T[k] -= s * std::pow(2.0 * kPi, n) * sgn;
  }
  T[0] += kPi / (a * a);
  // the 26 nearest images other than n = 0, removed from psi: + d^gamma (1/|x|)(n)
  ensure_derivs(q);
  Vec d(g_der.mi.size());
  for (int nz = -1; nz <= 1; ++nz)
    for (int ny = -1; ny <= 1; ++ny)
      for (int nx = -1; nx <= 1; ++nx) {
        if (!nx && !ny && !nz) continue;
        double x[3] = {(double)nx, (double)ny, (double)nz};
        g_der.inv_r(x, d.data());
        for (int k = 0; k < nq; ++k) T[k] += d[k];
      }
  return T;
}

// ---------------------------------------------------------------------------
// AMR hierarchy (Sec. 3): per level, leaf cells with masses and refined cells.
uint64_t morton(const I3& c, int lev) {
  uint64_t k = 0;
  for (int b = 0; b < lev; ++b) {
    k |= (uint64_t)((c[0] >> b) & 1) << (3 * b);
    k |= (uint64_t)((c[1] >> b) & 1) << (3 * b + 1);
    k |= (uint64_t)((c[2] >> b) & 1) << (3 * b + 2);
  }
  return k;
}
I3 parent_of(const I3& c) { return I3{c[0] >> 1, c[1] >> 1, c[2] >> 1}; }
void centre(const I3& c, int lev, double* x) {
  double h = std::ldexp(1.0, -lev);
  for (int i = 0; i < 3; ++i) x[i] = (c[i] + 0.5) * h;
}
I3 wrap(const I3& c, int lev) {  // the box holding image c (periodic)
  const int m = (1 << lev) - 1;
  return I3{c[0] & m, c[1] & m, c[2] & m};
}
bool inside(const I3& c, int lev) {
  int n = 1 << lev;
  return c[0] >= 0 && c[1] >= 0 && c[2] >= 0 && c[0] < n && c[1] < n && c[2] < n;
}

enum CellKind { OUTSIDE, ABSENT, LEAF, REFINED };

struct Hier {
  int lmin = 0, lmax = 0;
  std::vector<std::map<I3, int64_t>> leaf;  // level -> (ijk -> input index)
  std::vector<std::set<I3>> refined;        // level -> refined cells
  std::vector<std::vector<double>> mass;    // level -> masses by input index
  std::vector<std::vector<I3>> cells;       // level -> ijk by input index

  CellKind kind(int lev, const I3& c) const {
    if (!inside(c, lev)) return OUTSIDE;
    if (leaf[lev].count(c)) return LEAF;
    if (refined[lev].count(c)) return REFINED;
    return ABSENT;
  }
  double leaf_mass(int lev, const I3& c) const { return mass[lev][leaf[lev].at(c)]; }

  int build(int lmin_, int lmax_, const int64_t* n, const int32_t* const* ijk,
            const double* const* m, bool periodic = false) {
    lmin = lmin_;
    lmax = lmax_;
    if (lmin < 2 || lmax < lmin || lmax > 20) return ORC_ERR_ARG;
    leaf.assign(lmax + 1, {});
    refined.assign(lmax + 1, {});
    mass.assign(lmax + 1, {});
    cells.assign(lmax + 1, {});
    for (int l = lmin; l <= lmax; ++l) {
      int64_t nl = n[l - lmin];
      if (nl < 0) return ORC_ERR_ARG;
      mass[l].assign(m[l - lmin], m[l - lmin] + nl);
      for (int64_t i = 0; i < nl; ++i) {
        I3 c{ijk[l - lmin][3 * i], ijk[l - lmin][3 * i + 1], ijk[l - lmin][3 * i + 2]};
        if (!inside(c, l)) return ORC_ERR_OUT_OF_BOX;
        if (!leaf[l].emplace(c, i).second) return ORC_ERR_DUPLICATE;
        cells[l].push_back(c);
      }
    }
    // refined cells: parents of every existing cell one level finer
    for (int l = lmax - 1; l >= 0; --l) {
      for (const auto& kv : leaf[l + 1]) refined[l].insert(parent_of(kv.first));
      for (const auto& c : refined[l + 1]) refined[l].insert(parent_of(c));
    }
    for (int l = 0; l <= lmax; ++l)
      for (const auto& c : refined[l])
        if (leaf[l].count(c)) return ORC_ERR_DUPLICATE;
    // every refined cell has all 8 children (RAMSES octs), base level complete
    for (int l = 0; l < lmax; ++l)
      for (const auto& c : refined[l])
        for (int k = 0; k < 8; ++k) {
          I3 ch{2 * c[0] + (k & 1), 2 * c[1] + ((k >> 1) & 1), 2 * c[2] + ((k >> 2) & 1)};
          if (!leaf[l + 1].count(ch) && !refined[l + 1].count(ch)) return ORC_ERR_INCOMPLETE;
        }
    uint64_t nbase = (uint64_t)1 << (3 * lmin);
    if (leaf[lmin].size() + refined[lmin].size() != nbase) return ORC_ERR_INCOMPLETE;
    for (int l = 0; l < lmin; ++l)
      if (refined[l].size() != ((uint64_t)1 << (3 * l))) return ORC_ERR_INCOMPLETE;
    // graded rule (Sec. 3.2): a refined cell's father has all 3^3 neighbours refined
    for (int l = 1; l <= lmax; ++l)
      for (const auto& c : refined[l]) {
        I3 f = parent_of(c);
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              I3 nb{f[0] + dx, f[1] + dy, f[2] + dz};
              if (periodic) nb = wrap(nb, l - 1);  // the rule holds across the boundary too
              if (!inside(nb, l - 1)) continue;
              if (!refined[l - 1].count(nb)) return ORC_ERR_NOT_GRADED;
            }
      }
    return ORC_OK;
  }
};

// One FMM tree per AMR level (Sec. 3.1): tree[j][f] maps box ijk at FMM level f
// to the multipole of the level-j cells inside it, f = 1..j-1.
using Grid = std::map<I3, Vec>;
using Tree = std::vector<Grid>;

// BuildTree + Upward + CenterShift of Alg. 2 for tree j.  Moments are
// accumulated about each box's geometric centre directly, so CenterShift is
// the identity here.
Tree build_tree(const Hier& H, const Ops& op, int j) {
  Tree T(j);
  if (j < 2) return T;
  int nc = op.n();
  // P2M into the FMM grid one level above the AMR cells (Delta l = 1).
  for (const auto& kv : H.leaf[j]) {
    I3 b = parent_of(kv.first);
    double x[3], c[3];
    centre(kv.first, j, x);
    centre(b, j - 1, c);
    Vec& M = T[j - 1].emplace(b, Vec(nc, 0.0)).first->second;
    op.p2m(H.mass[j][kv.second], x, c, M);
  }
  // M2M up to FMM level 1.
  for (int f = j - 2; f >= 1; --f)
    for (const auto& kv : T[f + 1]) {
      I3 b = parent_of(kv.first);
      double cc[3], cp[3];
      centre(kv.first, f + 1, cc);
      centre(b, f, cp);
      Vec& M = T[f].emplace(b, Vec(nc, 0.0)).first->second;
      op.m2m(kv.second, cc, cp, M);
    }
  return T;
}

struct Solver {
  const Hier& H;
  int p;
  int bottom;               // 0: M2P bottom intermediate field (paper); 1: M2L into F + L2P
  int delta = 1;            // levels between the cells and the finest FMM box (2: unigrids only)
  bool periodic = false;    // images of the box everywhere (see the header); set by set_periodic
  Vec T;                    // lattice tensor, |gamma| <= p + 1
  Vec Mroot;                // multipole of every leaf about the box centre
  Ops op;
  std::vector<Tree> trees;  // indexed by AMR level j

  Solver(const Hier& h, int p_, int pm = 0, int bottom_ = 0) : H(h), p(p_), bottom(bottom_), op(p_, pm) {
    ensure_derivs(p + 1);
    trees.resize(H.lmax + 1);
    for (int j = H.lmin; j <= H.lmax; ++j) trees[j] = build_tree(H, op, j);
  }

  void set_periodic() {
    periodic = true;
    T = lattice_tensor(p + 1, 2.0);
    Mroot.assign(op.n(), 0.0);
    const double c0[3] = {0.5, 0.5, 0.5};
    for (int j = H.lmin; j <= H.lmax; ++j)
      for (const auto& kv : H.leaf[j]) {
        double x[3];
        centre(kv.first, j, x);
        op.p2m(H.mass[j][kv.second], x, c0, Mroot);
      }
  }
  // the box a (possibly image) index refers to, and whether it exists
  I3 W(const I3& c, int lev) const { return periodic ? wrap(c, lev) : c; }
  bool keep(const I3& c, int lev) const { return periodic || inside(c, lev); }

  // Multipole drifting of the stale trees j < lo (see the header): vel[j] holds
  // the velocity of each leaf of level j (input order), dt[j - lmin] the time
  // since level j was set.  Boxes whose tree mass is zero are not moved.
  void drift(int lo, const double* const* vel, const double* dt) {
    for (int j = H.lmin; j < lo && j <= H.lmax; ++j) {
      const double tj = dt[j - H.lmin];
      if (tj == 0.0 || !vel[j - H.lmin]) continue;
      for (int f = 1; f < j; ++f) {
        std::map<I3, std::array<double, 4>> mp;  // box -> (mass, momentum) of tree j
        for (const auto& kv : H.leaf[j]) {
          I3 b = kv.first;
          for (int s = j; s > f; --s) b = parent_of(b);
          const double m = H.mass[j][kv.second];
          const double* v = vel[j - H.lmin] + 3 * kv.second;
          auto& a = mp[b];
          a[0] += m;
          for (int i = 0; i < 3; ++i) a[1 + i] += m * v[i];
        }
        for (auto& kv : trees[j][f]) {
          auto it = mp.find(kv.first);
          if (it == mp.end() || it->second[0] == 0.0) continue;
          double c[3], cd[3];
          centre(kv.first, f, c);
          for (int i = 0; i < 3; ++i) cd[i] = c[i] - it->second[1 + i] / it->second[0] * tj;
          Vec out(op.n(), 0.0);
          op.m2m(kv.second, c, cd, out);  // moments about c - d of the unmoved mass
          kv.second = out;
        }
      }
    }
  }

  // RebuildMergedTree of Alg. 1: merged[f][box] = sum_{j>=l+1} M_{j;f}[box].
  std::vector<Grid> merged_tree(int l) const {
    std::vector<Grid> mt(H.lmax + 1);
    for (int j = l + 1; j <= H.lmax; ++j)
      for (int f = 1; f < j; ++f)
        for (const auto& kv : trees[j][f]) {
          Vec& M = mt[f].emplace(kv.first, Vec(op.n(), 0.0)).first->second;
          for (int k = 0; k < op.n(); ++k) M[k] += kv.second[k];
        }
    return mt;
  }

  const Vec* tree_box(int j, int f, const I3& b) const {
    if (j < H.lmin || j > H.lmax || f < 1 || f >= j) return nullptr;
    auto it = trees[j][f].find(b);
    return it == trees[j][f].end() ? nullptr : &it->second;
  }
  static const Vec* grid_box(const std::vector<Grid>& g, int f, const I3& b) {
    if (f < 0 || f >= (int)g.size()) return nullptr;
    auto it = g[f].find(b);
    return it == g[f].end() ? nullptr : &it->second;
  }

  // Interaction list of box B at level b (Sec. 2): children of the 3^3
  // neighbours of B's parent, minus the 3^3 neighbours of B, inside the box.
  // Periodic: the boxes are images (geometry), W() gives the box they show.
  std::vector<I3> ilist(const I3& B, int b) const {
    std::vector<I3> out;
    I3 P = parent_of(B);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          I3 Q{P[0] + dx, P[1] + dy, P[2] + dz};
          if (!keep(Q, b - 1)) continue;
          for (int k = 0; k < 8; ++k) {
            I3 S{2 * Q[0] + (k & 1), 2 * Q[1] + ((k >> 1) & 1), 2 * Q[2] + ((k >> 2) & 1)};
            if (std::abs(S[0] - B[0]) <= 1 && std::abs(S[1] - B[1]) <= 1 &&
                std::abs(S[2] - B[2]) <= 1)
              continue;
            out.push_back(S);
          }
        }
    return out;
  }

  // MultipoleToLocal (Alg. 3) for target level l: L at every level-b ancestor
  // (b = 2..top) of a level-l leaf, top = l-2 (bottom mode 1: l-1, the
  // parent box F itself).  Level 0 and 1 boxes have empty interaction lists,
  // so the first local expansion is at box level 2.
  std::vector<Grid> downward(int l, const std::vector<Grid>& mt, int nthreads) const {
    std::vector<Grid> L(l + 1);
    const int top = bottom ? l - 1 : l - 1 - delta;
    const int b0 = periodic ? 1 : 2;  // first level with an interaction list
    if (top < b0) return L;
    // boxes that need L: ancestors of level-l leaves
    std::vector<std::set<I3>> need(l + 1);
    for (const auto& kv : H.leaf[l]) {
      I3 c = kv.first;
      for (int b = l - 1; b >= b0; --b) {
        c = parent_of(c);
        if (b <= top) need[b].insert(c);
      }
    }
    int nc = op.n();
    // periodic: the root's local expansion from every image beyond its 3^3
    // (and the background): Eq. 3 with the lattice tensor, about the box centre
    Vec Lroot;
    const double c0[3] = {0.5, 0.5, 0.5};
    if (periodic) {
      Lroot.assign(nc, 0.0);
      op.m2l(Mroot, T, Lroot);
    }
    for (int b = b0; b <= top; ++b) {
      std::vector<I3> boxes(need[b].begin(), need[b].end());
      std::vector<Vec> res(boxes.size(), Vec(nc, 0.0));
#pragma omp parallel num_threads(nthreads)
      {
        DCache dc(p + 1);
#pragma omp for schedule(dynamic, 16)
        for (long ib = 0; ib < (long)boxes.size(); ++ib) {
          const I3& B = boxes[ib];
          Vec& Lb = res[ib];
          double cB[3];
          centre(B, b, cB);
          if (b > b0) {  // ShiftLocal of the parent's expansion (Eq. 4)
            I3 P = parent_of(B);
            double cP[3];
            centre(P, b - 1, cP);
            op.l2l(L[b - 1].at(P), cP, cB, Lb);
          } else if (periodic) {  // level 1: the root's lattice expansion
            op.l2l(Lroot, c0, cB, Lb);
          }
          for (const I3& Si : ilist(B, b)) {
            const I3 S = W(Si, b);  // content
            double cS[3], R[3];
            centre(Si, b, cS);  // geometry of the image
            for (int i = 0; i < 3; ++i) R[i] = cB[i] - cS[i];
            CellKind k = H.kind(b, S);
            if (k == LEAF) {  // tree j = b carries cell masses: P2L
              op.p2l(H.leaf_mass(b, S), dc.get(R), Lb);
              continue;
            }
            // trees j = b+1 .. min(l, lmax), then the merged tree (j >= l+1)
            for (int j = std::max(H.lmin, b + 1); j <= std::min(l, H.lmax); ++j)
              if (const Vec* M = tree_box(j, b, S)) op.m2l(*M, dc.get(R), Lb);
            if (l < H.lmax)
              if (const Vec* M = grid_box(mt, b, S)) op.m2l(*M, dc.get(R), Lb);
          }
        }
      }
      for (size_t ib = 0; ib < boxes.size(); ++ib) L[b][boxes[ib]] = res[ib];
    }
    return L;
  }

  // PotentialEvaluation with Delta l = 2 on a single complete level l: the
  // level l-2 ancestor G of the target is the finest FMM box.
  void evaluate_dl2(int l, const I3& t, const std::vector<Grid>& L, DCache& dc, double* phi,
                    double* grad) const {
    double xt[3];
    centre(t, l, xt);
    const I3 G = parent_of(parent_of(t));
    if (l - 3 >= 2) {  // far field: local expansion of G's parent (level l-3)
      const I3 P = parent_of(G);
      double c[3];
      centre(P, l - 3, c);
      op.l2p(L[l - 3].at(P), c, xt, phi, grad);
    }
    for (const I3& S : ilist(G, l - 2)) {  // intermediate field: M2P at level l-2
      double cS[3], R[3];
      centre(S, l - 2, cS);
      for (int i = 0; i < 3; ++i) R[i] = xt[i] - cS[i];
      if (const Vec* M = tree_box(l, l - 2, S)) op.m2p(*M, dc.get(R), phi, grad);
    }
    for (int dz = -1; dz <= 1; ++dz)  // near field: every cell of G's 3^3 neighbours
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const I3 N{G[0] + dx, G[1] + dy, G[2] + dz};
          if (!inside(N, l - 2)) continue;
          for (int k = 0; k < 64; ++k) {
            const I3 C{4 * N[0] + (k & 3), 4 * N[1] + ((k >> 2) & 3), 4 * N[2] + (k >> 4)};
            if (C == t) continue;
            double cC[3];
            centre(C, l, cC);
            p2p(H.leaf_mass(l, C), cC, xt, phi, grad);
          }
        }
  }

  // PotentialEvaluation (Alg. 4, with Fig. 2's list of sources) for one target.
  void evaluate(int l, const I3& t, const std::vector<Grid>& L, const std::vector<Grid>& mt,
                DCache& dc, double* phi, double* grad) const {
    if (delta == 2) {
      evaluate_dl2(l, t, L, dc, phi, grad);
      return;
    }
    double xt[3];
    centre(t, l, xt);
    I3 F = parent_of(t);
    if (bottom) {
      // bottom mode 1: far and intermediate fields both from F's local expansion
      if (l - 1 >= 2) {
        double c[3];
        centre(F, l - 1, c);
        op.l2p(L[l - 1].at(F), c, xt, phi, grad);
      }
    } else if (l - 2 >= (periodic ? 1 : 2)) {
      // far field: local expansion of the level l-2 box
      I3 G2 = parent_of(F);
      double c[3];
      centre(G2, l - 2, c);
      op.l2p(L[l - 2].at(G2), c, xt, phi, grad);
    }
    // intermediate field: interaction list of F at level l-1 (bottom mode 0)
    if (!bottom)
    for (const I3& Si : ilist(F, l - 1)) {
      const I3 S = W(Si, l - 1);
      double cS[3], R[3];
      centre(Si, l - 1, cS);
      CellKind k = H.kind(l - 1, S);
      if (k == LEAF) {  // (i) coarse leaves: P2P with their mass
        p2p(H.leaf_mass(l - 1, S), cS, xt, phi, grad);
        continue;
      }
      for (int i = 0; i < 3; ++i) R[i] = xt[i] - cS[i];
      if (const Vec* M = tree_box(l, l - 1, S)) op.m2p(*M, dc.get(R), phi, grad);  // (ii) T_l
      if (l < H.lmax)
        if (const Vec* M = grid_box(mt, l - 1, S)) op.m2p(*M, dc.get(R), phi, grad);  // (iii)
    }
    // near and nearest fields: the 3^3 neighbours of F
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          I3 N{F[0] + dx, F[1] + dy, F[2] + dz};
          CellKind kn = H.kind(l - 1, W(N, l - 1));
          if (kn == OUTSIDE) continue;
          double cN[3];
          centre(N, l - 1, cN);
          if (kn == LEAF) {  // a level l-1 leaf covers 8 positions: counted once
            p2p(H.leaf_mass(l - 1, W(N, l - 1)), cN, xt, phi, grad);
            continue;
          }
          if (kn != REFINED) { std::fprintf(stderr, "oracle: near cell absent\n"); continue; }
          for (int k = 0; k < 8; ++k) {
            I3 P{2 * N[0] + (k & 1), 2 * N[1] + ((k >> 1) & 1), 2 * N[2] + ((k >> 2) & 1)};
            if (P == t) continue;
            CellKind kp = H.kind(l, W(P, l));
            double cP[3];
            centre(P, l, cP);
            if (kp == LEAF) {
              p2p(H.leaf_mass(l, W(P, l)), cP, xt, phi, grad);
              continue;
            }
            bool touching = std::abs(P[0] - t[0]) <= 1 && std::abs(P[1] - t[1]) <= 1 &&
                            std::abs(P[2] - t[2]) <= 1;
            if (touching) {  // nearest field (Sec. 3.2): P2P from the 2^3 children
              for (int kc = 0; kc < 8; ++kc) {
                I3 C{2 * P[0] + (kc & 1), 2 * P[1] + ((kc >> 1) & 1), 2 * P[2] + ((kc >> 2) & 1)};
                if (H.kind(l + 1, W(C, l + 1)) != LEAF) {
                  std::fprintf(stderr, "oracle: nearest child not a leaf\n");
                  continue;
                }
                double cC[3];
                centre(C, l + 1, cC);
                p2p(H.leaf_mass(l + 1, W(C, l + 1)), cC, xt, phi, grad);
              }
            } else {  // near field refined cell: M2P from the merged tree at FMM level l
              double R[3] = {xt[0] - cP[0], xt[1] - cP[1], xt[2] - cP[2]};
              if (const Vec* M = grid_box(mt, l, W(P, l))) op.m2p(*M, dc.get(R), phi, grad);
            }
          }
        }
  }
};

}  // namespace

// ---------------------------------------------------------------------------
// C API (called from Python through ctypes by the tests and the benchmark).
extern "C" {

// Solve for the leaf cells of levels lo..lmax.  Inputs per level l = lmin..lmax
// at index l-lmin: n leaf cells, ijk int32[n][3], mass double[n].  sel/n_sel
// choose a subset of each level's leaves (indices into that level's input);
// n_sel == NULL means all leaves.  phi[l-lmin] (double[n_sel]) and
// acc[l-lmin] (double[n_sel][3]) receive G*phi and -G*grad phi.  Returns 0 or a
// negative validation code.
// p_m: multipole order of M2L / M2P (0: p); bottom: 0 = M2P, 1 = M2L + L2P.
// vel (per level, double [n][3], or NULL) and dt (per level, or NULL): drift
// the multipoles of the stale trees j < lo (see Solver::drift).
static int solve_impl(int lmin, int lmax, const int64_t* n, const int32_t* const* ijk,
                      const double* const* mass, int p, double G, int p_m, int bottom, int delta,
                      const double* const* vel, const double* dt, int lo,
                      const int64_t* n_sel, const int64_t* const* sel, double* const* phi,
                      double* const* acc, int nthreads, bool periodic = false) {
  if (p < 1 || p > 12 || nthreads < 1 || p_m < 0 || p_m > p || (bottom != 0 && bottom != 1)) return ORC_ERR_ARG;
  Hier H;
  int rc = H.build(lmin, lmax, n, ijk, mass, periodic);
  if (rc) return rc;
  if (lo < lmin || lo > lmax) return ORC_ERR_ARG;
  Solver S(H, p, p_m, bottom);
  S.delta = delta;
  if (periodic) S.set_periodic();
  if (vel && dt) S.drift(lo, vel, dt);
  for (int l = lo; l <= lmax; ++l) {
    int64_t nt = n_sel ? n_sel[l - lmin] : n[l - lmin];
    if (nt == 0) continue;
    std::vector<Grid> mt;
    if (l < lmax) mt = S.merged_tree(l);
    std::vector<Grid> L = S.downward(l, mt, nthreads);
#pragma omp parallel num_threads(nthreads)
    {
      DCache dc(p + 1);
#pragma omp for schedule(dynamic, 64)
      for (int64_t i = 0; i < nt; ++i) {
        int64_t idx = n_sel ? sel[l - lmin][i] : i;
        const I3& t = H.cells[l][idx];
        double ph = 0.0, gr[3] = {0.0, 0.0, 0.0};
        S.evaluate(l, t, L, mt, dc, &ph, gr);
        phi[l - lmin][i] = G * ph;
        for (int k = 0; k < 3; ++k) acc[l - lmin][3 * i + k] = -G * gr[k];
      }
    }
  }
  return ORC_OK;
}

int oracle_fmm_solve(int lmin, int lmax, const int64_t* n, const int32_t* const* ijk,
                     const double* const* mass, int p, double G, int p_m, int bottom,
                     const double* const* vel, const double* dt, int lo,
                     const int64_t* n_sel, const int64_t* const* sel, double* const* phi,
                     double* const* acc, int nthreads) {
  return solve_impl(lmin, lmax, n, ijk, mass, p, G, p_m, bottom, 1, vel, dt, lo, n_sel, sel, phi, acc, nthreads);
}

// The Delta l = 2 variant (see the header) on one complete level l = lmin =
// lmax >= 3; arguments as oracle_fmm_solve without the bottom mode, drifting
// and lo.
int oracle_fmm_solve_dl2(int level, const int64_t* n, const int32_t* const* ijk, const double* const* mass,
                         int p, double G, int p_m, const int64_t* n_sel, const int64_t* const* sel,
                         double* const* phi, double* const* acc, int nthreads) {
  if (level < 3) return ORC_ERR_ARG;
  if (n[0] != ((int64_t)1 << (3 * level))) return ORC_ERR_INCOMPLETE;
  return solve_impl(level, level, n, ijk, mass, p, G, p_m, 0, 2, nullptr, nullptr, level, n_sel, sel, phi, acc,
                    nthreads);
}

// Periodic boundaries (see the header), bottom M2P, lmin >= 3; arguments as
// oracle_fmm_solve without the bottom mode and drifting.
int oracle_fmm_solve_periodic(int lmin, int lmax, const int64_t* n, const int32_t* const* ijk,
                              const double* const* mass, int p, double G, int p_m, int lo,
                              const int64_t* n_sel, const int64_t* const* sel, double* const* phi,
                              double* const* acc, int nthreads) {
  if (lmin < 3) return ORC_ERR_ARG;
  return solve_impl(lmin, lmax, n, ijk, mass, p, G, p_m, 0, 1, nullptr, nullptr, lo, n_sel, sel, phi, acc,
                    nthreads, true);
}

// The periodic potential by Ewald's sum over all pairs (O(N^2 K)), with
// splitting parameter `alpha` (>= 6): phi_t = G (sum_{j != t} m_j psi(x_t - x_j)
// + m_t psi_self), accel_t = -G sum_{j != t} m_j grad psi(x_t - x_j).  The
// reciprocal part goes through the structure factors S(k) = sum_j m_j e^{2 pi i k.x_j}.
int oracle_ewald_sum(int lmin, int lmax, const int64_t* n, const int32_t* const* ijk, const double* const* mass,
                     double G, double alpha, int lo, const int64_t* n_sel, const int64_t* const* sel,
                     double* const* phi, double* const* acc, int nthreads) {
  if (nthreads < 1 || lmin < 0 || lmax < lmin || lo < lmin || lo > lmax || !(alpha >= 6.0)) return ORC_ERR_ARG;
  std::vector<double> X, M;
  for (int l = lmin; l <= lmax; ++l)
    for (int64_t i = 0; i < n[l - lmin]; ++i) {
      I3 c{ijk[l - lmin][3 * i], ijk[l - lmin][3 * i + 1], ijk[l - lmin][3 * i + 2]};
      double x[3];
      centre(c, l, x);
      X.insert(X.end(), x, x + 3);
      M.push_back(mass[l - lmin][i]);
    }
  const int64_t N = (int64_t)M.size();
  Ewald ew(alpha);
  const int64_t K = (int64_t)ew.kv.size();
  std::vector<double> Sre(K, 0.0), Sim(K, 0.0);
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int64_t q = 0; q < K; ++q) {
    double re = 0.0, im = 0.0;
    for (int64_t j = 0; j < N; ++j) {
      double ph = 2.0 * kPi * (ew.kv[q][0] * X[3 * j] + ew.kv[q][1] * X[3 * j + 1] + ew.kv[q][2] * X[3 * j + 2]);
      re += M[j] * std::cos(ph);
      im += M[j] * std::sin(ph);
    }
    Sre[q] = re;
    Sim[q] = im;
  }
  const double self = ew.self();
  for (int l = lo; l <= lmax; ++l) {
    int64_t nt = n_sel ? n_sel[l - lmin] : n[l - lmin];
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; ++i) {
      int64_t idx = n_sel ? sel[l - lmin][i] : i;
      I3 c{ijk[l - lmin][3 * idx], ijk[l - lmin][3 * idx + 1], ijk[l - lmin][3 * idx + 2]};
      double xt[3];
      centre(c, l, xt);
      double v = 0.0, g[3] = {0.0, 0.0, 0.0}, mself = 0.0;
      // real space: the 27 images of every other mass
      for (int64_t j = 0; j < N; ++j) {
        const double* y = &X[3 * j];
        if (y[0] == xt[0] && y[1] == xt[1] && y[2] == xt[2]) {
          mself += M[j];
          continue;
        }
        double r[3] = {xt[0] - y[0], xt[1] - y[1], xt[2] - y[2]};
        double vv = 0.0, gg[3] = {0.0, 0.0, 0.0};
        for (int nz = -1; nz <= 1; ++nz)
          for (int ny = -1; ny <= 1; ++ny)
            for (int nx = -1; nx <= 1; ++nx) {
              double x[3] = {r[0] + nx, r[1] + ny, r[2] + nz};
              ew.real(x, &vv, gg);
            }
        v += M[j] * vv;
        for (int k = 0; k < 3; ++k) g[k] += M[j] * gg[k];
      }
      // reciprocal space over all masses, then the target's own share removed
      // (its images enter through psi_self)
      double vr = 0.0, gr[3] = {0.0, 0.0, 0.0};
      for (int64_t q = 0; q < K; ++q) {
        const auto& k = ew.kv[q];
        double ph = 2.0 * kPi * (k[0] * xt[0] + k[1] * xt[1] + k[2] * xt[2]);
        double cs = std::cos(ph), sn = std::sin(ph);
        // sum_j m_j cos(2 pi k.(x - x_j)) = cos(k.x) Re S + sin(k.x) Im S
        vr += k[3] * (cs * Sre[q] + sn * Sim[q]);
        double d = k[3] * 2.0 * kPi * (-sn * Sre[q] + cs * Sim[q]);
        for (int a = 0; a < 3; ++a) gr[a] += d * k[a];
      }
      double recip_self = 0.0;
      for (int64_t q = 0; q < K; ++q) recip_self += ew.kv[q][3];
      vr -= mself * recip_self;
      double psi_sum = -(v + vr - kPi / (alpha * alpha) * (std::accumulate(M.begin(), M.end(), 0.0) - mself));
      phi[l - lmin][i] = G * (psi_sum + mself * self);
      for (int k = 0; k < 3; ++k) acc[l - lmin][3 * i + k] = G * (g[k] + gr[k]);
    }
  }
  return ORC_OK;
}

// The lattice tensor T_gamma, |gamma| <= q, multi-index order (see lattice_tensor).
void oracle_lattice_tensor(int q, double alpha, double* out) {
  Vec T = lattice_tensor(q, alpha);
  for (size_t k = 0; k < T.size(); ++k) out[k] = T[k];
}

// O(N^2) direct sum over all leaves of all levels (self term excluded), for
// the selected targets.  Same argument conventions as oracle_fmm_solve.
int oracle_direct_sum(int lmin, int lmax, const int64_t* n, const int32_t* const* ijk,
                      const double* const* mass, double G, int lo, const int64_t* n_sel,
                      const int64_t* const* sel, double* const* phi, double* const* acc,
                      int nthreads) {
  if (nthreads < 1 || lmin < 0 || lmax < lmin || lo < lmin || lo > lmax) return ORC_ERR_ARG;
  std::vector<double> X, M;
  for (int l = lmin; l <= lmax; ++l)
    for (int64_t i = 0; i < n[l - lmin]; ++i) {
      I3 c{ijk[l - lmin][3 * i], ijk[l - lmin][3 * i + 1], ijk[l - lmin][3 * i + 2]};
      double x[3];
      centre(c, l, x);
      X.insert(X.end(), x, x + 3);
      M.push_back(mass[l - lmin][i]);
    }
  int64_t N = (int64_t)M.size();
  for (int l = lo; l <= lmax; ++l) {
    int64_t nt = n_sel ? n_sel[l - lmin] : n[l - lmin];
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 64)
    for (int64_t i = 0; i < nt; ++i) {
      int64_t idx = n_sel ? sel[l - lmin][i] : i;
      I3 c{ijk[l - lmin][3 * idx], ijk[l - lmin][3 * idx + 1], ijk[l - lmin][3 * idx + 2]};
      double xt[3];
      centre(c, l, xt);
      double ph = 0.0, gr[3] = {0.0, 0.0, 0.0};
      for (int64_t s = 0; s < N; ++s) {
        const double* y = &X[3 * s];
        if (y[0] == xt[0] && y[1] == xt[1] && y[2] == xt[2]) continue;
        p2p(M[s], y, xt, &ph, gr);
      }
      phi[l - lmin][i] = G * ph;
      for (int k = 0; k < 3; ++k) acc[l - lmin][3 * i + k] = -G * gr[k];
    }
  }
  return ORC_OK;
}

// Canonical tree index for bit-exact comparison.  For each level l = 1..lmax:
// octs (the 8 children of a refined level l-1 cell) ordered by the Morton key
// of their parent cell (x in the lowest bit of each triple); cell id = 8*oct +
// (x&1 | (y&1)<<1 | (z&1)<<2).  Call with out arrays NULL to get n_oct[l]
// (int64[lmax+1]); then again with buffers:
//   oct_key[l]  uint64[n_oct]     Morton key of the parent cell at level l-1
//   status[l]   int64[8*n_oct]    refined: child oct id at l+1; leaf: -1 - input index
//   nbr[l]      int64[27*n_oct]   oct under the parent's neighbour (dx,dy,dz) at
//               index (dx+1)+3(dy+1)+9(dz+1); -2 - (cell id at l-1) when that
//               neighbour is a level l-1 leaf; -1 outside the unit box.
int oracle_tree(int lmin, int lmax, const int64_t* n, const int32_t* const* ijk,
                const double* const* mass, int64_t* n_oct, uint64_t* const* oct_key,
                int64_t* const* status, int64_t* const* nbr) {
  Hier H;
  int rc = H.build(lmin, lmax, n, ijk, mass);
  if (rc) return rc;
  // per level: octs sorted by parent Morton key
  std::vector<std::map<uint64_t, I3>> octs(lmax + 1);  // key -> parent ijk at l-1
  for (int l = 1; l <= lmax; ++l)
    for (const auto& P : H.refined[l - 1]) octs[l][morton(P, l - 1)] = P;
  for (int l = 0; l <= lmax; ++l) n_oct[l] = (l == 0) ? 0 : (int64_t)octs[l].size();
  if (!oct_key) return ORC_OK;
  auto oct_rank = [&](int l, const I3& P) -> int64_t {  // oct at level l whose parent is P
    auto it = octs[l].find(morton(P, l - 1));
    if (it == octs[l].end()) return -1;
    return (int64_t)std::distance(octs[l].begin(), it);
  };
  auto cell_id = [&](int l, const I3& c) -> int64_t {  // id of an existing level-l cell
    I3 P = parent_of(c);
    int64_t o = oct_rank(l, P);
    int pos = (c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2);
    return 8 * o + pos;
  };
  for (int l = 1; l <= lmax; ++l) {
    int64_t o = 0;
    for (const auto& kv : octs[l]) {
      const I3& P = kv.second;
      oct_key[l][o] = kv.first;
      for (int k = 0; k < 8; ++k) {
        I3 c{2 * P[0] + (k & 1), 2 * P[1] + ((k >> 1) & 1), 2 * P[2] + ((k >> 2) & 1)};
        int64_t s;
        if (H.kind(l, c) == LEAF)
          s = -1 - H.leaf[l].at(c);
        else
          s = (l < lmax) ? oct_rank(l + 1, c) : -1;
        status[l][8 * o + k] = s;
      }
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            I3 Q{P[0] + dx, P[1] + dy, P[2] + dz};
            int64_t v;
            CellKind k = H.kind(l - 1, Q);
            if (k == OUTSIDE)
              v = -1;
            else if (k == REFINED)
              v = oct_rank(l, Q);
            else if (k == LEAF)
              v = -2 - cell_id(l - 1, Q);
            else
              v = -1;  // absent: impossible for a graded hierarchy
            nbr[l][27 * o + (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] = v;
          }
      ++o;
    }
  }
  return ORC_OK;
}

// ---- unit access for the pins --------------------------------------------
int oracle_ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

void oracle_multi_index(int p, int32_t* abc) {
  MultiIndex mi;
  mi.build(p);
  for (int k = 0; k < mi.size(); ++k)
    for (int j = 0; j < 3; ++j) abc[3 * k + j] = mi.list[k][j];
}

// d^gamma(1/r) at R for |gamma| <= q, in multi-index order.
void oracle_inv_r_derivs(int q, const double* R, double* out) {
  ensure_derivs(q);
  int n = oracle_ncoef(q);
  std::vector<double> tmp(g_der.mi.size());
  g_der.inv_r(R, tmp.data());
  for (int k = 0; k < n; ++k) out[k] = tmp[k];
}

// Integer numerators P_gamma(u) of d^gamma(1/r) = P_gamma / r^(2|gamma|+1).
void oracle_numerators(int q, const int64_t* u, int64_t* out) {
  ensure_derivs(q);
  long long uu[3] = {u[0], u[1], u[2]};
  for (int k = 0; k < oracle_ncoef(q); ++k) out[k] = g_der.numerator(k, uu);
}

void oracle_p2m(int p, double m, const double* x, const double* c, double* M) {
  Ops op(p);
  Vec v(M, M + op.n());
  op.p2m(m, x, c, v);
  std::memcpy(M, v.data(), sizeof(double) * op.n());
}
void oracle_m2m(int p, const double* Mc, const double* cc, const double* cp, double* Mp) {
  Ops op(p);
  Vec a(Mc, Mc + op.n()), b(Mp, Mp + op.n());
  op.m2m(a, cc, cp, b);
  std::memcpy(Mp, b.data(), sizeof(double) * op.n());
}
void oracle_m2l(int p, const double* M, const double* cs, const double* ct, double* L) {
  ensure_derivs(p + 1);
  Ops op(p);
  DCache dc(p + 1);
  double R[3] = {ct[0] - cs[0], ct[1] - cs[1], ct[2] - cs[2]};
  Vec a(M, M + op.n()), b(L, L + op.n());
  op.m2l(a, dc.get(R), b);
  std::memcpy(L, b.data(), sizeof(double) * op.n());
}
void oracle_l2l(int p, const double* Lp, const double* cp, const double* cc, double* Lc) {
  Ops op(p);
  Vec a(Lp, Lp + op.n()), b(Lc, Lc + op.n());
  op.l2l(a, cp, cc, b);
  std::memcpy(Lc, b.data(), sizeof(double) * op.n());
}
void oracle_l2p(int p, const double* L, const double* c, const double* x, double* phi_grad) {
  Ops op(p);
  Vec a(L, L + op.n());
  op.l2p(a, c, x, &phi_grad[0], &phi_grad[1]);
}
void oracle_m2p(int p, const double* M, const double* cs, const double* x, double* phi_grad) {
  ensure_derivs(p + 1);
  Ops op(p);
  DCache dc(p + 1);
  double R[3] = {x[0] - cs[0], x[1] - cs[1], x[2] - cs[2]};
  Vec a(M, M + op.n());
  op.m2p(a, dc.get(R), &phi_grad[0], &phi_grad[1]);
}

int oracle_max_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
