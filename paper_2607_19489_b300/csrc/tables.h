// tables.h -- host-built, dimensionless translation operators of the FMM.
//
// All expansions on the device are stored in box units: a box of level b has
// size h = 2^-b, its multipole is kept as Mt_alpha = M_alpha / h^|alpha| and
// its local expansion as Lt_beta = L_beta * h^(|beta|+1).  With g(hR) =
// h^-(|g|+1) g(R) (g = -1/r is homogeneous of degree -1) every translation
// operator is then the same for all levels, so one table per operator serves
// the whole tree.
#pragma once
#include <array>
#include <cstdint>
#include <vector>

namespace fmm {

inline int ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// Graded multi-index order: degree n, then a descending, then b descending.
struct MultiIdx {
  int q = -1;
  std::vector<std::array<int, 3>> list;
  std::vector<int> lut;  // (q+1)^3 -> index or -1
  void build(int q);
  int at(int a, int b, int c) const {
    if (a < 0 || b < 0 || c < 0 || a > q || b > q || c > q) return -1;
    return lut[(a * (q + 1) + b) * (q + 1) + c];
  }
  int size() const { return (int)list.size(); }
};

// Integer numerators P_gamma(u) of d^gamma(1/r) = P_gamma(u)/|u|^(2|gamma|+1),
// |gamma| <= q, from the recurrence obtained by differentiating the identity
// r^2 d_i(1/r) + x_i (1/r) = 0 (exact, 128-bit integers).
void inv_r_numerators(int q, const int64_t u[3], std::vector<__int128>& P, const MultiIdx& mi);

// The 26 neighbour offsets of a box other than itself, as 27-indices
// (dx+1)+3(dy+1)+9(dz+1).
extern const int kNbr26[26];

struct Tables {
  int p = 0, nc = 0, nc1 = 0;  // ncoef(p), ncoef(p+1)
  int pm = 0;                  // multipole order of M2L / M2P / near M2P (<= p): terms with
                               // |alpha| > pm are zero in those operators (Eq. 3 with
                               // multipoles up to order pm only)
  MultiIdx mi;                 // |alpha| <= p+1

  // Operators (FP64).  Index conventions:
  //  f, t, s, b, c in 0..7 are child positions x | y<<1 | z<<2 inside an oct.
  //  qi in 0..25 indexes kNbr26.
  // M2P, bottom intermediate field (Fig. 2): rows of the source oct-level
  // (l-1) grid; output n = (f*8+t)*4+comp for the target cell t of cell f,
  // comp 0 = phi, 1..3 = accel (-grad phi); input k = (qi*8+s)*nc + alpha.
  std::vector<double> m2p;  // [256][26*8*nc]
  // M2L (Eq. 3): output n = b*nc + beta, input as above.
  std::vector<double> m2l;  // [8*nc][26*8*nc]
  // Near-field M2P from a refined cell at integer offset R = target - source
  // (level-l units), R in [-3,3]^3: [343][nc][4].
  std::vector<double> nearop;
  // L2P from the level l-2 box to the 64 grandchild cell centres:
  // [64 = f*8+t][nc][4].
  std::vector<double> l2p;
  // M2M (Eq. 2) as pair lists per output alpha: input gamma, child sign
  // pattern e (bit i = parity of alpha_i - gamma_i) and coefficient.
  std::vector<int> m2m_off, m2m_g, m2m_e;
  std::vector<double> m2m_c;
  // L2L (Eq. 4) as pair lists per output beta: input gamma, sign pattern e,
  // coefficient.
  std::vector<int> l2l_off, l2l_off8, l2l_g, l2l_e;
  std::vector<double> l2l_c;
  // degree of each coefficient (|alpha|) for alpha < nc
  std::vector<int> degree;

  // Delta l = 2 (footnote of Sec. 2; unigrids), built by build_dl2():
  // M2P from the interaction list of the level l-2 box G: rows of the level
  // l-2 grid, output n = ((g*8+f)*8+t)*4+comp for target t of cell f of the
  // child oct of cell g, input k = (qi*8+s)*nc + alpha; results in level l-1
  // units (the accumulator's).
  std::vector<double> m2p2;  // [2048][26*8*nc]
  // the near-field ring: P2P from the level-l children of the level l-1 cells
  // in the interaction list of the target's parent F (inside the 12^3 near
  // field of Delta l = 2 but outside Delta l = 1's 6^3): rows of the level l-1
  // grid, output as m2p, input k = (qi*8+s)*8 + child; level l-1 units.
  std::vector<double> p2pr;  // [256][26*64]

  // Periodic boundaries: the local expansions of the 8 level-1 boxes (box
  // units) from their multipoles (box units): through the root, from every
  // image of the root beyond its 3^3 and the neutralising background (M2M to
  // the root, the lattice M2L = Eq. 3 with D = the lattice tensor, L2L back
  // down), plus the level-1 M2L from the root's 26 nearest images (built
  // after m2l).  lattice[(c nc + beta) 8 nc + c' nc + alpha].
  std::vector<double> lattice;

  void build(int p, int p_m = 0);  // p_m = 0: p
  void build_dl2();
  void build_lattice();
};

// The lattice tensor T_gamma = d^gamma psi_far(0), |gamma| <= q, in the order
// of mi: psi_far = Ewald's periodic potential of a unit mass with its uniform
// neutralising background (box [0,1)^3, g = -1/r) minus g over the 27 images
// n in {-1,0,1}^3.
std::vector<double> lattice_tensor(int q, const MultiIdx& mi);

}  // namespace fmm
