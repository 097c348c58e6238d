// Plain double-precision CPU reference ("oracle") of the wall-modelled lattice Boltzmann LES step.
//
// TEST INFRASTRUCTURE ONLY. This file is the independent checker for the CUDA path: it shares no
// code, header, table or helper with it. Only tests, the smoke check and the benchmark's CPU
// baseline may load it. The product path never calls it.
//
// It is deliberately slow and literal: two population arrays (pre-collision state F, post-collision
// state P), a collide loop followed by a pull-stream loop, every quantity computed from its
// definition in double precision. Nothing is blocked, fused or reordered.
//
// What it follows (Kummerländer et al., "Large-Scale Simulations of Turbulent Flows using Lattice
// Boltzmann Methods on Heterogeneous High Performance Computers"):
//   * velocity set D3Q19 (Sec. 2.2, Fig. "lattice"); D3Q27 as the same construction with 27 speeds;
//   * the homogenised LB update of Eq. (hlbm) with the BGK reading f^(1) = f - f^eq(rho,u);
//   * the second-order equilibrium (the n<=2 part of the Hermite equilibrium of Sec. 2.2);
//   * the convex homogenised velocity of Eq. (convexVelocity), porosity given per cell as
//     gamma = 1 - d (gamma = 1: fluid);
//   * the Smagorinsky effective relaxation time of Eq. (tauEff) with Eqs. (sgsStress),(turbVisc);
//   * the Spalding wall function of Eq. (spaldingfunct) with the normalisations Eqs. (u+),(y+),
//     entering as the solid velocity u^B with the finite-difference (sigma = 0) non-equilibrium
//     part (Sec. 2.2.1);
//   * a regularised local velocity inlet (Sec. 2.2.2, last paragraph) and a fixed local pressure
//     outlet and full-slip outer faces (Sec. 3.2);
//   * the hybrid recursive regularised collision of Sec. 2.2 (third-order Hermite equilibrium,
//     recursive third-order f^(1), finite-difference strain) as the alternative collision model;
//   * the vortex-method turbulent inlet of Sec. 2.2.2 and the porous-medium inputs of Sec. 2.1
//     (Forchheimer permeability, Eq. lattice_porosity);
//   * the GLUPs definition of Sec. 3.1 is not computed here (it is a timing quantity).
// Readings where the paper is silent or garbled are stated next to the code that takes them.
//
// The discrete adjoint exported at the end is the transpose of this oracle's own step, built from
// per-cell Jacobians obtained by forward-mode dual numbers (no hand-derived reverse formulas).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdio>
#include <vector>
#include <string>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------------------------
// Dual numbers (value, derivative) for forward-mode differentiation of the per-cell update.
struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual operator+(double a, Dual b) { return Dual(a) + b; }
inline Dual operator+(Dual a, double b) { return a + Dual(b); }
inline Dual operator-(double a, Dual b) { return Dual(a) - b; }
inline Dual operator-(Dual a, double b) { return a - Dual(b); }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, Dual b) { return Dual(a) / b; }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  // d sqrt(x) at x = 0 is taken as 0 (the one-sided subgradient of |Pi| at Pi = 0).
  return Dual(s, s > 0.0 ? a.d / (2.0 * s) : 0.0);
}
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, e * a.d); }
inline Dual log(Dual a) { return Dual(std::log(a.v), a.d / a.v); }
inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }
using std::sqrt; using std::exp; using std::log;

// ---------------------------------------------------------------------------------------------
// Velocity sets. Ordering: i = 0 is the rest velocity; for D3Q19 the pairs (i, i+9), i = 1..9,
// are opposite; for D3Q27 the pairs (i, i+13), i = 1..13. Weights follow from |c|^2 (Sec. 2.2,
// Fig. "lattice" for D3Q19): D3Q19 1/3, 1/18, 1/36; D3Q27 8/27, 2/27, 1/54, 1/216.
struct Lat {
  int Q = 0;
  int c[27][3] = {};
  double w[27] = {};
  int W[27] = {};      // integer weights (w * Wden), used for the wall normal sums
  int Wden = 1;
  int opp[27] = {};
};

Lat make_lattice(int q) {
  Lat L;
  L.Q = q;
  int half[13][3];
  int nh = 0;
  // The first half of the moving speeds, in the documented order.
  const int base[13][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1},
                           {0, 1, 1}, {0, 1, -1}, {1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
  nh = (q == 19) ? 9 : 13;
  for (int k = 0; k < nh; ++k)
    for (int a = 0; a < 3; ++a) half[k][a] = base[k][a];
  for (int a = 0; a < 3; ++a) L.c[0][a] = 0;
  for (int k = 0; k < nh; ++k)
    for (int a = 0; a < 3; ++a) {
      L.c[1 + k][a] = half[k][a];
      L.c[1 + nh + k][a] = -half[k][a];
    }
  for (int i = 0; i < q; ++i) {
    int n2 = L.c[i][0] * L.c[i][0] + L.c[i][1] * L.c[i][1] + L.c[i][2] * L.c[i][2];
    if (q == 19) {
      const int Wi[3] = {12, 2, 1};
      L.Wden = 36;
      L.W[i] = Wi[n2];
    } else {
      const int Wi[4] = {64, 16, 4, 1};
      L.Wden = 216;
      L.W[i] = Wi[n2];
    }
    L.w[i] = double(L.W[i]) / double(L.Wden);
  }
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j)
      if (L.c[j][0] == -L.c[i][0] && L.c[j][1] == -L.c[i][1] && L.c[j][2] == -L.c[i][2]) L.opp[i] = j;
  return L;
}

int dir_index(const Lat& L, int cx, int cy, int cz) {
  for (int i = 0; i < L.Q; ++i)
    if (L.c[i][0] == cx && L.c[i][1] == cy && L.c[i][2] == cz) return i;
  return -1;
}

constexpr double CS2 = 1.0 / 3.0;  // lattice speed of sound squared

enum { M_FLUID = 0, M_SOLID = 1, M_INFLOW = 3, M_OUTFLOW = 4 };                  // mask input codes
enum { K_FLUID = 0, K_SOLID = 1, K_WALL = 2, K_INFLOW = 3, K_OUTFLOW = 4 };         // classified kinds
enum { F_PERIODIC = 0, F_WALL = 1, F_SLIP = 2, F_OPEN = 3 };                       // face kinds

struct Oracle {
  Lat L;
  int nx = 0, ny = 0, nz = 0;
  long N = 0;
  double tau0 = 0.6, cs = 0.0;
  int face[6] = {F_PERIODIC, F_PERIODIC, F_PERIODIC, F_PERIODIC, F_PERIODIC, F_PERIODIC};
  std::vector<uint8_t> mask;
  std::vector<double> ywall;
  std::vector<uint8_t> kind, isref;
  std::vector<int> nsum;      // 3 per cell: integer wall-normal sums (WALL cells)
  std::vector<long> refcell;  // per cell: reference cell of a WALL cell, or -1
  double force[3] = {0, 0, 0};
  std::vector<double> uin;    // 3 * ny * nz, component-major: uin[a*ny*nz + y + ny*z]
  double rho_out = 1.0;
  std::vector<double> gamma;  // N, empty means 1 everywhere
  bool wm = false;
  double kappa = 0.41, E = 9.52;
  int storage = 0;            // 0 exact, 1 fp32, 2 fp16, 3 bf16 rounding of stored f - w
  int model = 0;              // collision: 0 BGK, 1 hybrid recursive regularised (HRR)
  double sigma = 1.0;         // HRR hybridisation factor (1: local stress only)
  std::vector<double> F, P, Fn;
  std::vector<double> uref_prev, uref_cur;
  std::vector<double> uvel_prev, uvel_cur;  // 3N component-major: velocity field of the last step (HRR)
  // vortex-method inlet (Sec. 2.2.2); off when vm_n == 0
  int vm_n = 0;
  double vm_sigma = 4.0, vm_I = 0.1;
  uint64_t vm_seed = 0;
  std::vector<double> uin_cur;  // inlet velocity of the current (last) step, 3 * ny * nz
  // outlet fringe zone (Sec. 3.2); off when fr_L == 0
  // sub-domain of a z-slab decomposition: the first gh_lo and last gh_hi z-planes are ghost planes
  // (cells owned by the neighbouring sub-domains): classified like every cell, never collided or
  // streamed, filled by the halo exchange
  int gh_lo = 0, gh_hi = 0;
  int fr_L = 0;
  int fr_x0 = 0;  // first plane of the layer (nx - L for the whole domain; any value for a crop)
  double fr_smax = 0.0, fr_p = 2.0;
  long t = 0;
  // adjoint bookkeeping
  std::vector<std::vector<double>> hist;  // stored pre-collision states S_0..S_{T-1}
  std::vector<std::vector<double>> href;  // stored reference-velocity buffers per step
  std::vector<double> dJdS_w;             // per-cell weight of d J / d rho at window steps
  long T_run = 0, W_run = 0;
};

std::string g_err;

inline long idx(const Oracle& o, int x, int y, int z) { return long(x) + long(o.nx) * (long(y) + long(o.ny) * long(z)); }
inline void coords(const Oracle& o, long n, int& x, int& y, int& z) {
  x = int(n % o.nx);
  long r = n / o.nx;
  y = int(r % o.ny);
  z = int(r / o.ny);
}

// Wrap a position across periodic faces. Returns a bit mask of the non-periodic faces that the
// position lies beyond: bit 2a for coordinate < 0 on axis a, bit 2a+1 for coordinate >= n_a.
int resolve(const Oracle& o, int p[3]) {
  const int dims[3] = {o.nx, o.ny, o.nz};
  int crossed = 0;
  for (int a = 0; a < 3; ++a) {
    if (p[a] < 0) {
      if (o.face[2 * a] == F_PERIODIC) p[a] += dims[a];
      else crossed |= 1 << (2 * a);
    } else if (p[a] >= dims[a]) {
      if (o.face[2 * a + 1] == F_PERIODIC) p[a] -= dims[a];
      else crossed |= 1 << (2 * a + 1);
    }
  }
  return crossed;
}

bool any_face_of_kind(const Oracle& o, int crossed, int k) {
  for (int f = 0; f < 6; ++f)
    if ((crossed >> f & 1) && o.face[f] == k) return true;
  return false;
}
bool all_faces_of_kind(const Oracle& o, int crossed, int k) {
  for (int f = 0; f < 6; ++f)
    if ((crossed >> f & 1) && o.face[f] != k) return false;
  return true;
}

// A neighbour position counts as solid if it is a SOLID cell, or lies beyond a bounce-back face.
bool solid_like(const Oracle& o, int x, int y, int z, const int d[3]) {
  int p[3] = {x + d[0], y + d[1], z + d[2]};
  int crossed = resolve(o, p);
  if (crossed) return any_face_of_kind(o, crossed, F_WALL);
  return o.mask[idx(o, p[0], p[1], p[2])] == M_SOLID;
}

// A cell "next to the boundary": some streaming source x - c_i is a SOLID cell or lies beyond a
// non-periodic face.
bool near_boundary(const Oracle& o, long r) {
  int x, y, z;
  coords(o, r, x, y, z);
  for (int i = 1; i < o.L.Q; ++i) {
    int q[3] = {x - o.L.c[i][0], y - o.L.c[i][1], z - o.L.c[i][2]};
    if (resolve(o, q)) return true;
    if (o.mask[idx(o, q[0], q[1], q[2])] == M_SOLID) return true;
  }
  return false;
}

// Cell classification: kind precedence SOLID > INFLOW > OUTFLOW > WALL > FLUID, where WALL is a
// non-solid cell with at least one solid(-like) neighbour. Wall normal n = -v/|v| with
// v = sum over solid neighbours of w_i c_i (integer weights). Reference cell of a WALL cell: the
// cell one step from it along the dominant axis of n (ties: lowest axis), provided that cell is a
// FLUID cell away from every boundary (no solid or outside streaming source). Reading of Sec. 2.2.1:
// the wall law's reference point has to lie in the flow; in gaps one or two cells wide it would sit
// on the opposite wall or on a domain face, and such a WALL cell has no reference (u^B = 0).
void classify(Oracle& o) {
  const Lat& L = o.L;
  o.kind.assign(o.N, K_FLUID);
  o.isref.assign(o.N, 0);
  o.nsum.assign(3 * o.N, 0);
  o.refcell.assign(o.N, -1);
  for (long n = 0; n < o.N; ++n) {
    int x, y, z;
    coords(o, n, x, y, z);
    uint8_t m = o.mask[n];
    if (m == M_SOLID) { o.kind[n] = K_SOLID; continue; }
    if (m == M_INFLOW) { o.kind[n] = K_INFLOW; continue; }
    if (m == M_OUTFLOW) { o.kind[n] = K_OUTFLOW; continue; }
    bool wall = false;
    int v[3] = {0, 0, 0};
    for (int i = 1; i < L.Q; ++i) {
      if (solid_like(o, x, y, z, L.c[i])) {
        wall = true;
        for (int a = 0; a < 3; ++a) v[a] += L.W[i] * L.c[i][a];
      }
    }
    if (wall) {
      o.kind[n] = K_WALL;
      for (int a = 0; a < 3; ++a) o.nsum[3 * n + a] = v[a];
    }
  }
  for (long n = 0; n < o.N; ++n) {
    if (o.kind[n] != K_WALL) continue;
    const int* v = &o.nsum[3 * n];
    if (v[0] == 0 && v[1] == 0 && v[2] == 0) continue;
    int a = 0;
    for (int b = 1; b < 3; ++b)
      if (std::abs(v[b]) > std::abs(v[a])) a = b;
    int x, y, z;
    coords(o, n, x, y, z);
    int p[3] = {x, y, z};
    p[a] += (v[a] > 0) ? -1 : 1;  // along n = -v
    if (resolve(o, p)) continue;
    long r = idx(o, p[0], p[1], p[2]);
    if (o.kind[r] != K_FLUID || near_boundary(o, r)) continue;
    o.refcell[n] = r;
    o.isref[r] = 1;
  }
}

// Source of the population f_i arriving at non-solid cell n after streaming: the post-collision
// population j of cell m, i.e. f_i(x, t+1) = f*_j(x_m, t). Rules (reading of Sec. 2.2 and 3.2):
//   * neighbour x - c_i inside (after periodic wrap) and not solid: (i, x - c_i);
//   * neighbour solid: half-way bounce-back, (opp(i), x);
//   * neighbour beyond an open (inflow/outflow) face: unknown; filled with the bounce-back value
//     (opp(i), x) and replaced by the boundary condition of the cell;
//   * neighbour beyond full-slip faces only: specular reflection, the population that left the
//     partner cell (x - c_i with the crossed coordinates set back to x's) with the crossed
//     velocity components reversed; bounce-back if that partner is solid;
//   * neighbour beyond a bounce-back face: (opp(i), x).
void source(const Oracle& o, long n, int i, int& j, long& m) {
  const Lat& L = o.L;
  int x, y, z;
  coords(o, n, x, y, z);
  int p[3] = {x - L.c[i][0], y - L.c[i][1], z - L.c[i][2]};
  int crossed = resolve(o, p);
  if (!crossed) {
    long s = idx(o, p[0], p[1], p[2]);
    if (o.mask[s] == M_SOLID) { j = L.opp[i]; m = n; }
    else { j = i; m = s; }
    return;
  }
  if (any_face_of_kind(o, crossed, F_OPEN) || !all_faces_of_kind(o, crossed, F_SLIP)) {
    j = L.opp[i]; m = n;
    return;
  }
  const int xs[3] = {x, y, z};
  int cj[3] = {L.c[i][0], L.c[i][1], L.c[i][2]};
  for (int a = 0; a < 3; ++a)
    if (crossed >> (2 * a) & 3) { p[a] = xs[a]; cj[a] = -cj[a]; }
  long s = idx(o, p[0], p[1], p[2]);
  if (o.mask[s] == M_SOLID) { j = L.opp[i]; m = n; return; }
  j = dir_index(L, cj[0], cj[1], cj[2]);
  m = s;
}

// Second-order equilibrium f_i^eq = w_i rho (1 + c.u/cs^2 + (c.u)^2/(2 cs^4) - u.u/(2 cs^2)).
template <class T>
T feq(const Lat& L, int i, T rho, const T u[3]) {
  T cu = double(L.c[i][0]) * u[0] + double(L.c[i][1]) * u[1] + double(L.c[i][2]) * u[2];
  T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return L.w[i] * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

// Q_i : A with Q_i = c_i c_i - cs^2 I (the second Hermite polynomial), A symmetric 3x3.
template <class T>
T q_contract(const Lat& L, int i, const T A[3][3]) {
  T s = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double q = double(L.c[i][a] * L.c[i][b]) - (a == b ? CS2 : 0.0);
      s = s + q * A[a][b];
    }
  return s;
}

// ---- Third-order Hermite terms of the HRR collision (Sec. 2.2) ---------------------------------
// Third-order Hermite polynomial H_abc(c) = c_a c_b c_c - cs^2 (c_a d_bc + c_b d_ac + c_c d_ab).
// With unit speeds H_aaa = c_a (c_a^2 - 1) vanishes on both velocity sets, which leaves the six
// mixed polynomials H_aab (a != b) and H_xyz; H_xyz vanishes on D3Q19 (no speed has three non-zero
// components) and is dropped there. Reading of the third-order terms of the equilibrium and of
// f^(1): a symmetric rank-3 tensor a enters as the weighted combination of the remaining
// polynomials whose lattice moments sum_i (.) H_k(c_i) equal the components a_k, i.e.
//   t_i = w_i sum_{k,l} H_k(c_i) (G^{-1})_{kl} a_l,   G_{kl} = sum_i w_i H_k(c_i) H_l(c_i).
// Where G is diagonal (D3Q27: G = 2 cs^6 for the mixed, cs^6 for H_xyz) this is the Hermite term
// H^(3) : a / (6 cs^6) of the expansion; on D3Q19 the mixed polynomials are not orthogonal and the
// Gram inverse gives the projection onto what the velocity set carries.
struct Third {
  int n = 0;
  int idx[7][3] = {};
  double P[7][27] = {};
  double Ginv[7][7] = {};
};

double hermite3(const Lat& L, int i, int a, int b, int c) {
  const int* v = L.c[i];
  return double(v[a] * v[b] * v[c]) - CS2 * (double(v[a]) * (b == c) + double(v[b]) * (a == c) + double(v[c]) * (a == b));
}

Third make_third(const Lat& L) {
  Third t;
  const int cand[7][3] = {{0, 0, 1}, {0, 0, 2}, {1, 1, 0}, {1, 1, 2}, {2, 2, 0}, {2, 2, 1}, {0, 1, 2}};
  for (int k = 0; k < 7; ++k) {
    double nrm = 0.0;
    double vals[27];
    for (int i = 0; i < L.Q; ++i) {
      vals[i] = hermite3(L, i, cand[k][0], cand[k][1], cand[k][2]);
      nrm += vals[i] * vals[i];
    }
    if (nrm == 0.0) continue;
    for (int a = 0; a < 3; ++a) t.idx[t.n][a] = cand[k][a];
    for (int i = 0; i < L.Q; ++i) t.P[t.n][i] = vals[i];
    ++t.n;
  }
  // Gram matrix and its inverse by Gauss-Jordan elimination with partial pivoting
  double G[7][14] = {};
  for (int k = 0; k < t.n; ++k) {
    for (int l = 0; l < t.n; ++l) {
      double s = 0.0;
      for (int i = 0; i < L.Q; ++i) s += L.w[i] * t.P[k][i] * t.P[l][i];
      G[k][l] = s;
    }
    G[k][t.n + k] = 1.0;
  }
  for (int col = 0; col < t.n; ++col) {
    int piv = col;
    for (int r = col + 1; r < t.n; ++r)
      if (std::fabs(G[r][col]) > std::fabs(G[piv][col])) piv = r;
    for (int m = 0; m < 2 * t.n; ++m) std::swap(G[col][m], G[piv][m]);
    const double d = G[col][col];
    for (int m = 0; m < 2 * t.n; ++m) G[col][m] /= d;
    for (int r = 0; r < t.n; ++r) {
      if (r == col) continue;
      const double fct = G[r][col];
      for (int m = 0; m < 2 * t.n; ++m) G[r][m] -= fct * G[col][m];
    }
  }
  for (int k = 0; k < t.n; ++k)
    for (int l = 0; l < t.n; ++l) t.Ginv[k][l] = G[k][t.n + l];
  return t;
}

const Third& third_of(const Lat& L) {
  static const Third t19 = make_third(make_lattice(19));
  static const Third t27 = make_third(make_lattice(27));
  return L.Q == 19 ? t19 : t27;
}

// w_i-weighted third-order term of population i for the symmetric tensor a (a[a][b][c]).
template <class T>
T third_term(const Lat& L, int i, const T a[3][3][3]) {
  const Third& t = third_of(L);
  T s = 0.0;
  for (int k = 0; k < t.n; ++k)
    for (int l = 0; l < t.n; ++l) s = s + (t.P[k][i] * t.Ginv[k][l]) * a[t.idx[l][0]][t.idx[l][1]][t.idx[l][2]];
  return L.w[i] * s;
}

// Third-order equilibrium of Sec. 2.2: the second-order one plus the third Hermite term with
// a_0^(3) = rho u u u.
template <class T>
T feq3(const Lat& L, int i, T rho, const T u[3]) {
  T a3[3][3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) a3[a][b][c] = rho * u[a] * u[b] * u[c];
  return feq(L, i, rho, u) + third_term(L, i, a3);
}

// Hybrid recursive regularised update (Eq. hlbm with the Hermite expansion of f^(1), Sec. 2.2):
//   f*_i = f^eq_i(rho, ueq) + (1 - 1/tau) f^(1)_i,
//   f^(1)_i = w_i Q_i : A2 / (2 cs^4) + third-order term of A3,
//   A3_abc = uh_a A2_bc + uh_b A2_ac + uh_c A2_ab (recursive third-order coefficient),
// with A2 the (hybridised) second-order non-equilibrium coefficient and uh the homogenised
// velocity around which f^(1) is expanded.
template <class T>
void collide_hrr(const Lat& L, T rho, const T ueq[3], const T uh[3], T tau, const T A2[3][3], T fs[27]) {
  T A3[3][3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) A3[a][b][c] = uh[a] * A2[b][c] + uh[b] * A2[a][c] + uh[c] * A2[a][b];
  for (int i = 0; i < L.Q; ++i) {
    T f1 = L.w[i] * q_contract(L, i, A2) / (2.0 * CS2 * CS2) + third_term(L, i, A3);
    fs[i] = feq3(L, i, rho, ueq) + (1.0 - 1.0 / tau) * f1;
  }
}

// Regularised boundary reconstruction (Latt et al.): given rho, u on the boundary and the known
// populations (unknown ones are those for which known[i] is false), set f^neq of each unknown
// population to that of its opposite, form Pi^neq = sum_i c_i c_i f^neq_i and replace every
// population by f^eq_i + w_i/(2 cs^4) Q_i : Pi^neq.
template <class T>
void regularise(const Lat& L, T f[27], T rho, const T u[3], const bool known[27]) {
  T fne[27];
  for (int i = 0; i < L.Q; ++i) fne[i] = f[i] - feq(L, i, rho, u);
  for (int i = 0; i < L.Q; ++i)
    if (!known[i]) fne[i] = fne[L.opp[i]];
  T Pi[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      T s = 0.0;
      for (int i = 0; i < L.Q; ++i) s = s + double(L.c[i][a] * L.c[i][b]) * fne[i];
      Pi[a][b] = s;
    }
  for (int i = 0; i < L.Q; ++i) f[i] = feq(L, i, rho, u) + L.w[i] / (2.0 * CS2 * CS2) * q_contract(L, i, Pi);
}

// Velocity inlet at a cell whose inward normal is +x: unknown populations have c_x > 0.
// rho from mass conservation across the face: rho (1 - u_x) = sum_{c_x=0} f + 2 sum_{c_x<0} f.
template <class T>
void bc_velocity(const Lat& L, T f[27], const T ub[3]) {
  T s0 = 0.0, sm = 0.0;
  bool known[27];
  for (int i = 0; i < L.Q; ++i) {
    known[i] = L.c[i][0] <= 0;
    if (L.c[i][0] == 0) s0 = s0 + f[i];
    if (L.c[i][0] < 0) sm = sm + f[i];
  }
  T rho = (s0 + 2.0 * sm) / (1.0 - ub[0]);
  regularise(L, f, rho, ub, known);
}

// Pressure outlet at a cell whose inward normal is -x: unknown populations have c_x < 0.
// rho = rho_out, u_x from rho_out (1 + u_x) = sum_{c_x=0} f + 2 sum_{c_x>0} f, tangential u = 0.
template <class T>
void bc_pressure(const Lat& L, T f[27], double rho_out) {
  T s0 = 0.0, sp = 0.0;
  bool known[27];
  for (int i = 0; i < L.Q; ++i) {
    known[i] = L.c[i][0] >= 0;
    if (L.c[i][0] == 0) s0 = s0 + f[i];
    if (L.c[i][0] > 0) sp = sp + f[i];
  }
  T rho = T(rho_out);
  T ub[3] = {-1.0 + (s0 + 2.0 * sp) / rho, T(0.0), T(0.0)};
  regularise(L, f, rho, ub, known);
}

// Effective relaxation time, Eq. (tauEff): tau_eff = nu_eff/cs^2 + 1/2, nu_eff = nu_mo + nu_turb,
// nu_turb = (C_S dx)^2 |S| (Eq. turbVisc), |S| = sqrt(2 S:S), with S recovered from the
// non-equilibrium stress S = -Pi^neq / (2 rho cs^2 tau_eff). Substituting gives a quadratic in
// tau_eff whose positive root is tau = (tau0 + sqrt(tau0^2 + 18 sqrt(2) C_S^2 |Pi|/rho)) / 2.
template <class T>
T tau_smagorinsky(double tau0, double cs, const T Pi[3][3], T rho) {
  T pp = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) pp = pp + Pi[a][b] * Pi[a][b];
  T pn = sqrt(pp);
  return 0.5 * (tau0 + sqrt(tau0 * tau0 + 18.0 * std::sqrt(2.0) * cs * cs * pn / rho));
}

// Spalding's law, Eq. (spaldingfunct): y+ = u+ + (1/E)[e^{k u+} - 1 - k u+ - (k u+)^2/2 - (k u+)^3/6].
double spalding_yplus(double up, double kappa, double E) {
  double k = kappa * up;
  return up + (std::exp(k) - 1.0 - k - k * k / 2.0 - k * k * k / 6.0) / E;
}
double spalding_dyplus(double up, double kappa, double E) {
  double k = kappa * up;
  return 1.0 + kappa * (std::exp(k) - 1.0 - k - k * k / 2.0) / E;
}

// Solve u+ * yplus(u+) = Re (the reference point's u_t y / nu) for u+ by Newton's method.
// The left side is increasing and convex in u+ >= 0, so Newton from a start at or right of the
// root converges monotonically. Start: sqrt(Re) (always right of the root since yplus(u) >= u),
// replaced by ln(2 E Re)/kappa when that is smaller and still right of the root.
double solve_uplus_from_re(double Re, double kappa, double E, int* iters) {
  if (!(Re > 0.0)) { if (iters) *iters = 0; return 0.0; }
  double u = std::sqrt(Re);
  if (kappa * u > 10.0) {
    double u1 = std::log(2.0 * E * Re) / kappa;
    if (u1 < u && u1 * spalding_yplus(u1, kappa, E) - Re >= 0.0) u = u1;
  }
  int k = 0;
  for (; k < 50; ++k) {
    double h = u * spalding_yplus(u, kappa, E) - Re;
    double dh = spalding_yplus(u, kappa, E) + u * spalding_dyplus(u, kappa, E);
    double du = h / dh;
    u -= du;
    if (std::fabs(du) <= 1e-14 * std::fabs(u)) { ++k; break; }
  }
  if (iters) *iters = k;
  return u;
}

// Solve yplus(u+) = yp for u+ (inverse of Spalding's law), Newton from the right as above.
double solve_uplus_from_yplus(double yp, double kappa, double E, int* iters) {
  if (!(yp > 0.0)) { if (iters) *iters = 0; return 0.0; }
  double u = yp;
  if (kappa * u > 10.0) {
    double u1 = std::log(2.0 * E * yp) / kappa;
    if (u1 < u && spalding_yplus(u1, kappa, E) - yp >= 0.0) u = u1;
  }
  int k = 0;
  for (; k < 50; ++k) {
    double h = spalding_yplus(u, kappa, E) - yp;
    double du = h / spalding_dyplus(u, kappa, E);
    u -= du;
    if (std::fabs(du) <= 1e-14 * std::fabs(u)) { ++k; break; }
  }
  if (iters) *iters = k;
  return u;
}

// Wall-model quantities of a WALL cell (Sec. 2.2.1; readings): tangential reference velocity
// u_t = u_r - (u_r.n) n at distance y_r = y_w + 1 from the wall, u_tau from Spalding at the
// reference point, u+ at the wall cell distance y_w, solid velocity u^B = u_tau u+_w t,
// modelled shear du/dn = (u_tau^2/nu) / (dy+/du+)(u+_w).
struct WallState { double uB[3]; double dudn; double t[3]; double n[3]; };

WallState wall_state(const Oracle& o, long n, const double* uref) {
  WallState ws{};
  const int* v = &o.nsum[3 * n];
  double vn = std::sqrt(double(v[0]) * v[0] + double(v[1]) * v[1] + double(v[2]) * v[2]);
  if (vn == 0.0 || o.refcell[n] < 0) return ws;
  for (int a = 0; a < 3; ++a) ws.n[a] = -double(v[a]) / vn;
  const double* ur = &uref[3 * o.refcell[n]];
  double un = ur[0] * ws.n[0] + ur[1] * ws.n[1] + ur[2] * ws.n[2];
  double ut[3];
  for (int a = 0; a < 3; ++a) ut[a] = ur[a] - un * ws.n[a];
  double U = std::sqrt(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
  if (U < 1e-12) return ws;
  for (int a = 0; a < 3; ++a) ws.t[a] = ut[a] / U;
  double nu = CS2 * (o.tau0 - 0.5);
  double yw = o.ywall.empty() ? 0.5 : o.ywall[n];
  double yr = yw + 1.0;
  double upr = solve_uplus_from_re(U * yr / nu, o.kappa, o.E, nullptr);
  double utau = U / upr;
  double upw = solve_uplus_from_yplus(yw * utau / nu, o.kappa, o.E, nullptr);
  for (int a = 0; a < 3; ++a) ws.uB[a] = utau * upw * ws.t[a];
  ws.dudn = (utau * utau / nu) / spalding_dyplus(upw, o.kappa, o.E);
  return ws;
}

// Finite-difference rate of strain S^FD (Sec. 2.2, non-local part of the hybrid f^(1)) at cell n
// from the velocity field of the previous step. Reading: a neighbour x +- e_b is usable when it lies
// inside the domain (after periodic wrap) and is not SOLID; the derivative d u_a / d x_b is the
// central difference when both are usable, the one-sided difference with the cell itself when one
// is, and zero when neither is. S = (grad u + grad u^T) / 2.
void strain_fd(const Oracle& o, long n, double S[3][3]) {
  int x, y, z;
  coords(o, n, x, y, z);
  const int here[3] = {x, y, z};
  double g[3][3];
  for (int b = 0; b < 3; ++b) {
    long nb[2] = {-1, -1};
    for (int s = 0; s < 2; ++s) {
      int p[3] = {here[0], here[1], here[2]};
      p[b] += s == 0 ? 1 : -1;
      if (resolve(o, p) != 0) continue;
      long m = idx(o, p[0], p[1], p[2]);
      if (o.kind[m] == K_SOLID) continue;
      nb[s] = m;
    }
    for (int a = 0; a < 3; ++a) {
      const double* u = o.uvel_prev.data() + long(a) * o.N;
      if (nb[0] >= 0 && nb[1] >= 0) g[a][b] = 0.5 * (u[nb[0]] - u[nb[1]]);
      else if (nb[0] >= 0) g[a][b] = u[nb[0]] - u[n];
      else if (nb[1] >= 0) g[a][b] = u[n] - u[nb[1]];
      else g[a][b] = 0.0;
    }
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) S[a][b] = 0.5 * (g[a][b] + g[b][a]);
}

// One cell's update. f holds the gathered pre-collision populations (boundary substitutions done);
// on return fs holds the post-collision populations, urep the reported velocity
// u = j/rho + F/(2 rho) and rho_out the density.
template <class T>
void collide_cell_core(const Oracle& o, long n, T f[27], T gamma, const T ub[3], const double* uref, T fs[27],
                       T urep[3], T* rho_out) {
  const Lat& L = o.L;
  int k = o.kind[n];
  if (k == K_INFLOW) bc_velocity(L, f, ub);
  if (k == K_OUTFLOW) bc_pressure(L, f, o.rho_out);
  T rho = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < L.Q; ++i) {
    rho = rho + f[i];
    for (int a = 0; a < 3; ++a) j[a] = j[a] + double(L.c[i][a]) * f[i];
  }
  T u[3];
  for (int a = 0; a < 3; ++a) {
    u[a] = j[a] / rho;
    urep[a] = u[a] + o.force[a] / (2.0 * rho);
  }
  if (rho_out) *rho_out = rho;
  if (k == K_WALL && o.wm) {
    // sigma = 0: the non-equilibrium part is the finite-difference one built from the modelled
    // strain S = (du/dn)/2 (t n^T + n t^T), f^(1,FD)_i = -(w_i rho tau/cs^2) Q_i : S; the
    // homogenised velocity is the solid velocity u^B (d = 1); |S| = |du/dn|.
    WallState ws = wall_state(o, n, uref);
    T S[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) S[a][b] = T(0.5 * ws.dudn * (ws.t[a] * ws.n[b] + ws.n[a] * ws.t[b]));
    double nu0 = CS2 * (o.tau0 - 0.5);
    double nut = o.cs * o.cs * std::fabs(ws.dudn);
    double tau = (nu0 + nut) / CS2 + 0.5;
    T uh[3];
    for (int a = 0; a < 3; ++a) uh[a] = ws.uB[a] + o.force[a] / rho;
    if (o.model == 1) {
      // HRR form: third-order equilibrium at u^B, f^(1) from A2 = -2 rho cs^2 tau S expanded
      // recursively around u^B.
      T A2[3][3], ub3[3];
      for (int a = 0; a < 3; ++a) {
        ub3[a] = T(ws.uB[a]);
        for (int b = 0; b < 3; ++b) A2[a][b] = -2.0 * CS2 * tau * rho * S[a][b];
      }
      collide_hrr(L, rho, uh, ub3, T(tau), A2, fs);
      return;
    }
    for (int i = 0; i < L.Q; ++i) {
      T f1 = -(L.w[i] * rho * tau / CS2) * q_contract(L, i, S);
      fs[i] = feq(L, i, rho, uh) + (1.0 - 1.0 / tau) * f1;
    }
    return;
  }
  T fe[27];
  for (int i = 0; i < L.Q; ++i) fe[i] = feq(L, i, rho, u);
  T Pi[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      T s = 0.0;
      for (int i = 0; i < L.Q; ++i) s = s + double(L.c[i][a] * L.c[i][b]) * (f[i] - fe[i]);
      Pi[a][b] = s;
    }
  T tau = (o.cs > 0.0) ? tau_smagorinsky(o.tau0, o.cs, Pi, rho) : T(o.tau0);
  // Eq. (convexVelocity) with gamma = 1 - d and u^B = 0 away from WALL cells; the body force enters
  // through the exact-difference shift u_hat += F/rho.
  T uh[3];
  for (int a = 0; a < 3; ++a) uh[a] = gamma * u[a] + o.force[a] / rho;
  if (o.model == 1) {
    // HRR: A2 = sigma Pi^neq + (1 - sigma) Pi^FD with Pi^FD = -2 rho cs^2 tau S^FD (the
    // Chapman-Enskog stress of the finite-difference strain; reading of the sign and of the missing
    // weight in the printed f^(1,FD)), expanded around the homogenised velocity gamma u.
    double Sfd[3][3];
    strain_fd(o, n, Sfd);
    T A2[3][3], uhom[3];
    for (int a = 0; a < 3; ++a) {
      uhom[a] = gamma * u[a];
      for (int b = 0; b < 3; ++b) A2[a][b] = o.sigma * Pi[a][b] + (1.0 - o.sigma) * (-2.0 * CS2) * tau * rho * Sfd[a][b];
    }
    collide_hrr(L, rho, uh, uhom, tau, A2, fs);
    return;
  }
  for (int i = 0; i < L.Q; ++i) fs[i] = feq(L, i, rho, uh) + (1.0 - 1.0 / tau) * (f[i] - fe[i]);
}

// Outlet fringe zone (Sec. 3.2: the outlet is a fixed local pressure with a fringe zone in front
// of it; the paper gives no parameters, so the layer is a reading). The last L planes x >= x0 =
// nx - L form the layer; in it every cell that is neither INFLOW nor OUTFLOW relaxes its
// post-collision populations towards the equilibrium at the outlet density and its own reported
// velocity:
//   f*_i <- f*_i - s(x) (f*_i - f^eq_i(rho_out, u)),   s(x) = s_max xi^p,  xi = (x - x0 + 1)/L,
// so the strength rises from s_max L^-p at the first plane to s_max at the last (p = 0: constant).
// (A crop of a larger domain keeps the domain's layer by giving its own x0.)
double fringe_strength(const Oracle& o, int x) {
  if (o.fr_L <= 0 || x < o.fr_x0) return 0.0;
  const double xi = double(x - o.fr_x0 + 1) / double(o.fr_L);
  return o.fr_smax * std::pow(xi, o.fr_p);
}

// One cell's update: the collision of collide_cell_core, then the fringe-zone relaxation.
template <class T>
void collide_cell(const Oracle& o, long n, T f[27], T gamma, const T ub[3], const double* uref, T fs[27],
                  T urep[3], T* rho_out) {
  collide_cell_core<T>(o, n, f, gamma, ub, uref, fs, urep, rho_out);
  const int k = o.kind[n];
  if (o.fr_L <= 0 || k == K_INFLOW || k == K_OUTFLOW) return;
  int x, y, z;
  coords(o, n, x, y, z);
  const double sx = fringe_strength(o, x);
  if (sx == 0.0) return;
  for (int i = 0; i < o.L.Q; ++i) fs[i] = fs[i] - sx * (fs[i] - feq(o.L, i, T(o.rho_out), urep));
}

double round_storage(int mode, double x);

void store_round(Oracle& o, std::vector<double>& A) {
  if (o.storage == 0) return;
  for (int i = 0; i < o.L.Q; ++i)
    for (long n = 0; n < o.N; ++n) {
      double& v = A[long(i) * o.N + n];
      v = o.L.w[i] + round_storage(o.storage, v - o.L.w[i]);
    }
}

void inlet_velocity(const Oracle& o, long n, double ub[3]) {
  int x, y, z;
  coords(o, n, x, y, z);
  long p = long(y) + long(o.ny) * z, pl = long(o.ny) * o.nz;
  const std::vector<double>& src = o.vm_n > 0 ? o.uin_cur : o.uin;
  for (int a = 0; a < 3; ++a) ub[a] = src.empty() ? 0.0 : src[a * pl + p];
}

double gamma_at(const Oracle& o, long n) { return o.gamma.empty() ? 1.0 : o.gamma[n]; }

// Reported moments of the state A (pre-collision, natural layout): boundary reconstruction at
// INFLOW/OUTFLOW cells, then rho = sum f, u = j/rho + F/(2 rho). SOLID cells report 0.
void moments_of(const Oracle& o, const std::vector<double>& A, double* rho, double* u) {
  const Lat& L = o.L;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < o.N; ++n) {
    if (o.kind[n] == K_SOLID) {
      rho[n] = 0.0;
      for (int a = 0; a < 3; ++a) u[a * o.N + n] = 0.0;
      continue;
    }
    double f[27];
    for (int i = 0; i < L.Q; ++i) f[i] = A[long(i) * o.N + n];
    double ub[3];
    inlet_velocity(o, n, ub);
    if (o.kind[n] == K_INFLOW) bc_velocity(L, f, ub);
    if (o.kind[n] == K_OUTFLOW) bc_pressure(L, f, o.rho_out);
    double r = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < L.Q; ++i) {
      r += f[i];
      for (int a = 0; a < 3; ++a) j[a] += L.c[i][a] * f[i];
    }
    rho[n] = r;
    for (int a = 0; a < 3; ++a) u[a * o.N + n] = j[a] / r + o.force[a] / (2.0 * r);
  }
}

void vm_reset(Oracle& o);

void init_refs(Oracle& o) {
  vm_reset(o);
  std::vector<double> rho(o.N), u(3 * o.N);
  moments_of(o, o.F, rho.data(), u.data());
  o.uref_prev.assign(3 * o.N, 0.0);
  for (long n = 0; n < o.N; ++n)
    if (o.isref[n])
      for (int a = 0; a < 3; ++a) o.uref_prev[3 * n + a] = u[a * o.N + n];
  o.uref_cur = o.uref_prev;
  o.uvel_prev = u;
  o.uvel_cur = u;
}

// ---- Vortex-method turbulent inlet (Sec. 2.2.2) ------------------------------------------------
// Counter-based random numbers: the SplitMix64 output function (Steele, Lea, Flood 2014) applied to
// seed + (1 + counter) * 0x9E3779B97F4A7C15, the top 53 bits scaled to [0, 1). Counter of vortex i,
// component c (0: y, 1: z, 2: sign) at step t: (t * n + i) * 4 + c.
uint64_t splitmix64_out(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double vm_uniform(uint64_t seed, uint64_t counter) {
  const uint64_t r = splitmix64_out(seed + (counter + 1) * 0x9E3779B97F4A7C15ull);
  return double(r >> 11) * (1.0 / 9007199254740992.0);
}

struct Vortex { double y, z, gamma; };

// Seed points of step t: positions uniform on the inlet plane [-1/2, ny - 1/2) x [-1/2, nz - 1/2)
// (cell centres at integer coordinates), signs +-1, circulation from the turbulent kinetic energy
// k_i = 3/2 (|u_mean(p_i)| I)^2 at the cell containing p_i:
//   Gamma_i = 4 s_i sqrt(pi k_i A / ((6 ln 3 - 9 ln 2) n)),  A = number of INFLOW cells.
std::vector<Vortex> vm_vortices(const Oracle& o, long t) {
  std::vector<Vortex> v(o.vm_n);
  long area = 0;
  for (long n = 0; n < o.N; ++n) area += o.kind[n] == K_INFLOW;
  const long pl = long(o.ny) * o.nz;
  for (int i = 0; i < o.vm_n; ++i) {
    const uint64_t base = (uint64_t(t) * uint64_t(o.vm_n) + uint64_t(i)) * 4ull;
    const double y = -0.5 + o.ny * vm_uniform(o.vm_seed, base + 0);
    const double z = -0.5 + o.nz * vm_uniform(o.vm_seed, base + 1);
    const double sg = vm_uniform(o.vm_seed, base + 2) < 0.5 ? 1.0 : -1.0;
    int iy = int(std::floor(y + 0.5)), iz = int(std::floor(z + 0.5));
    iy = std::min(std::max(iy, 0), o.ny - 1);
    iz = std::min(std::max(iz, 0), o.nz - 1);
    const long p = iy + long(o.ny) * iz;
    double um2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double ua = o.uin.empty() ? 0.0 : o.uin[a * pl + p];
      um2 += ua * ua;
    }
    const double k = 1.5 * um2 * o.vm_I * o.vm_I;
    const double gam = 4.0 * sg * std::sqrt(M_PI * k * double(area) / ((6.0 * std::log(3.0) - 9.0 * std::log(2.0)) * o.vm_n));
    v[i] = {y, z, gam};
  }
  return v;
}

// In-plane velocity induced at plane position (y, z) by the vortices, inflow direction d = +x:
//   u_v = (1/2pi) sum_i Gamma_i ((p_i - x) x d) (1 - e^{-a}) e^{-a} / |p_i - x|^2,  a = |p_i - x|^2/(2 sigma^2)
// (reading: the vortex profile whose energy integral gives the constant 6 ln 3 - 9 ln 2 of Gamma;
// the printed kernel has lost the sign of the exponent and the second factor). With r = p_i - x in
// the plane, r x e_x = (0, r_z, -r_y).
void vm_field(const std::vector<Vortex>& v, double sigma, double y, double z, double& uy, double& uz) {
  uy = 0.0;
  uz = 0.0;
  for (const Vortex& q : v) {
    const double ry = q.y - y, rz = q.z - z;
    const double r2 = ry * ry + rz * rz;
    if (r2 == 0.0) continue;
    const double e = std::exp(-r2 / (2.0 * sigma * sigma));
    const double f = q.gamma * (1.0 - e) * e / (2.0 * M_PI * r2);
    uy += f * rz;
    uz -= f * ry;
  }
}

// Inlet velocity of step t: u = u_mean + u_v + u'_x e_x with the streamwise fluctuation of the
// linear kinematic (Langevin) model, u'_x = -(u_v . grad U)/|grad U|, U the streamwise component of
// the previous step's inlet velocity (reading of the printed cross product as this projection);
// grad U by central differences over the plane positions, one-sided at the plane edges; u'_x = 0
// where grad U = 0.
void vm_update(Oracle& o, long t) {
  const std::vector<Vortex> v = vm_vortices(o, t);
  const long pl = long(o.ny) * o.nz;
  std::vector<double> next(3 * pl, 0.0);
  for (int z = 0; z < o.nz; ++z)
    for (int y = 0; y < o.ny; ++y) {
      const long p = y + long(o.ny) * z;
      double uy, uz;
      vm_field(v, o.vm_sigma, double(y), double(z), uy, uz);
      auto U = [&](int yy, int zz) { return o.uin_cur[yy + long(o.ny) * zz]; };
      double gy = 0.0, gz = 0.0;
      if (o.ny > 1) {
        if (y == 0) gy = U(1, z) - U(0, z);
        else if (y == o.ny - 1) gy = U(y, z) - U(y - 1, z);
        else gy = 0.5 * (U(y + 1, z) - U(y - 1, z));
      }
      if (o.nz > 1) {
        if (z == 0) gz = U(y, 1) - U(y, 0);
        else if (z == o.nz - 1) gz = U(y, z) - U(y, z - 1);
        else gz = 0.5 * (U(y, z + 1) - U(y, z - 1));
      }
      const double gn = std::sqrt(gy * gy + gz * gz);
      const double ux = gn > 0.0 ? -(uy * gy + uz * gz) / gn : 0.0;
      const double um[3] = {o.uin.empty() ? 0.0 : o.uin[p], o.uin.empty() ? 0.0 : o.uin[pl + p],
                            o.uin.empty() ? 0.0 : o.uin[2 * pl + p]};
      next[p] = um[0] + ux;
      next[pl + p] = um[1] + uy;
      next[2 * pl + p] = um[2] + uz;
    }
  o.uin_cur = next;
}

void vm_reset(Oracle& o) {
  o.uin_cur = o.uin;
  if (o.uin_cur.empty()) o.uin_cur.assign(3L * o.ny * o.nz, 0.0);
}

inline bool is_ghost(const Oracle& o, long n) {
  if (o.gh_lo == 0 && o.gh_hi == 0) return false;
  const long z = n / (long(o.nx) * o.ny);
  return z < o.gh_lo || z >= o.nz - o.gh_hi;
}

// One time step in two phases. Collide: every non-solid cell of F into P, recording the reference
// velocities. Stream: pull P into F through the source map. Between the two, a sub-domain of a slab
// decomposition receives the post-collision populations of its ghost cells that stream into it and
// the reference velocities its wall cells read next step (the halo exchange).
void step_collide(Oracle& o) {
  const Lat& L = o.L;
  if (o.vm_n > 0) vm_update(o, o.t);
#pragma omp parallel for schedule(static)
  for (long n = 0; n < o.N; ++n) {
    if (o.kind[n] == K_SOLID || is_ghost(o, n)) {
      for (int i = 0; i < L.Q; ++i) o.P[long(i) * o.N + n] = 0.0;
      continue;
    }
    double f[27], fs[27], urep[3], ub[3], rho;
    for (int i = 0; i < L.Q; ++i) f[i] = o.F[long(i) * o.N + n];
    inlet_velocity(o, n, ub);
    collide_cell<double>(o, n, f, gamma_at(o, n), ub, o.uref_prev.data(), fs, urep, &rho);
    for (int i = 0; i < L.Q; ++i) o.P[long(i) * o.N + n] = fs[i];
    if (o.isref[n])
      for (int a = 0; a < 3; ++a) o.uref_cur[3 * n + a] = urep[a];
    for (int a = 0; a < 3; ++a) o.uvel_cur[long(a) * o.N + n] = urep[a];
  }
}

void step_stream(Oracle& o) {
  const Lat& L = o.L;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < o.N; ++n) {
    for (int i = 0; i < L.Q; ++i) {
      if (o.kind[n] == K_SOLID || is_ghost(o, n)) { o.Fn[long(i) * o.N + n] = 0.0; continue; }
      int j; long m;
      source(o, n, i, j, m);
      o.Fn[long(i) * o.N + n] = o.P[long(j) * o.N + m];
    }
  }
  std::swap(o.F, o.Fn);
  store_round(o, o.F);
  o.uref_prev = o.uref_cur;
  o.uvel_prev = o.uvel_cur;
  ++o.t;
}

void step_once(Oracle& o) {
  step_collide(o);
  step_stream(o);
}

// Halo lists of one side of a sub-domain (side 0: the z- cut, side 1: the z+ cut). With zr the real
// boundary plane and zg the adjacent ghost plane, and an entry (p, pos) meaning population slot p of
// the plane cell at pos = x + nx y (the population opp(p) in transit, stored as in the in-place
// scheme's slot p):
//   list 0: the post-collision populations of cells of zr that stream into non-solid cells of zg
//           (the populations that leave through the cut);
//   list 1: the populations of cells of zg that stream into non-solid cells of zr (they come in);
//   list 2: pos of the cells of zr that a WALL cell of zg takes as reference cell;
//   list 3: pos of the cells of zg that a WALL cell of zr takes as reference cell.
// Entries run over pos ascending, then p ascending. The neighbour's list 1 (resp. 3) on the other
// side of the same cut equals this list 0 (resp. 2).
std::vector<long> halo_list(const Oracle& o, int side, int list) {
  std::vector<long> out;
  const long nxy = long(o.nx) * o.ny;
  const int zr = side == 0 ? o.gh_lo : o.nz - o.gh_hi - 1;
  const int zg = side == 0 ? o.gh_lo - 1 : o.nz - o.gh_hi;
  if ((side == 0 ? o.gh_lo : o.gh_hi) == 0) return out;
  if (list == 0 || list == 1) {
    // the populations that cross: f_i(n, t+1) = f*_j(m, t) with n on one side of the cut and m on
    // the other (streaming, bounce-back and slip rules of `source`), entered as (opp(j), pos(m))
    const int zn = list == 0 ? zg : zr;  // receiving plane
    const int zm = list == 0 ? zr : zg;  // plane of the sending cells
    std::vector<std::pair<long, int>> e;
    for (long pos = 0; pos < nxy; ++pos) {
      const long n = pos + nxy * zn;
      if (o.kind[n] == K_SOLID) continue;
      for (int i = 0; i < o.L.Q; ++i) {
        int j;
        long m;
        source(o, n, i, j, m);
        if (m / nxy == zm) e.emplace_back(m - nxy * zm, o.L.opp[j]);
      }
    }
    std::sort(e.begin(), e.end());
    for (const auto& v : e) out.push_back(long(v.second) * nxy + v.first);
    return out;
  }
  const int zw = list == 2 ? zg : zr;  // plane of the wall cells
  const int zt = list == 2 ? zr : zg;  // plane of their reference cells
  std::vector<uint8_t> hit(nxy, 0);
  for (long pos = 0; pos < nxy; ++pos) {
    const long w = pos + nxy * zw;
    if (o.kind[w] != K_WALL || o.refcell[w] < 0) continue;
    const long r = o.refcell[w];
    if (r / nxy == zt) hit[r - nxy * zt] = 1;
  }
  for (long pos = 0; pos < nxy; ++pos)
    if (hit[pos]) out.push_back(pos);
  return out;
}

// ---- 16-bit codecs written from the IEEE 754 binary16 and the bfloat16 definitions ------------
// Round-to-nearest-even of a double to the target format (nearbyint rounds ties to even in the
// default rounding mode; the scalings by powers of two are exact).
uint16_t f16_encode(double x) {
  uint16_t s = std::signbit(x) ? 0x8000 : 0;
  if (std::isnan(x)) return 0x7E00;
  double a = std::fabs(x);
  if (a >= 65520.0) return s | 0x7C00;
  if (a < std::ldexp(1.0, -14)) return s | uint16_t(std::nearbyint(std::ldexp(a, 24)));
  int e;
  std::frexp(a, &e);
  int E = e - 1;
  double q = std::nearbyint(std::ldexp(a, 10 - E));
  if (q == 2048.0) { q = 1024.0; ++E; }
  if (E > 15) return s | 0x7C00;
  return s | uint16_t((E + 15) << 10) | uint16_t(q - 1024.0);
}
double f16_decode(uint16_t b) {
  double s = (b & 0x8000) ? -1.0 : 1.0;
  int e = (b >> 10) & 31, m = b & 1023;
  if (e == 0) return s * std::ldexp(double(m), -24);
  if (e == 31) return m ? NAN : s * INFINITY;
  return s * std::ldexp(double(1024 + m), e - 25);
}
uint16_t bf16_encode(double x) {
  uint16_t s = std::signbit(x) ? 0x8000 : 0;
  if (std::isnan(x)) return 0x7FC0;
  double a = std::fabs(x);
  if (a >= std::ldexp(2.0 - std::ldexp(1.0, -8), 127)) return s | 0x7F80;
  if (a < std::ldexp(1.0, -126)) return s | uint16_t(std::nearbyint(std::ldexp(a, 133)));
  int e;
  std::frexp(a, &e);
  int E = e - 1;
  double q = std::nearbyint(std::ldexp(a, 7 - E));
  if (q == 256.0) { q = 128.0; ++E; }
  if (E > 127) return s | 0x7F80;
  return s | uint16_t((E + 127) << 7) | uint16_t(q - 128.0);
}
double bf16_decode(uint16_t b) {
  double s = (b & 0x8000) ? -1.0 : 1.0;
  int e = (b >> 7) & 255, m = b & 127;
  if (e == 0) return s * std::ldexp(double(m), -133);
  if (e == 255) return m ? NAN : s * INFINITY;
  return s * std::ldexp(double(128 + m), e - 134);
}
double round_storage(int mode, double x) {
  if (mode == 1) return double(float(x));
  if (mode == 2) return f16_decode(f16_encode(x));
  if (mode == 3) return bf16_decode(bf16_encode(x));
  return x;
}

// ---- adjoint helpers ----------------------------------------------------------------------------
// Per-cell Jacobian-transpose product: given mu (sensitivities of the post-collision populations of
// cell n), return lam_k = sum_j mu_j d fs_j / d f_k, and the sensitivities with respect to gamma(n)
// and the inlet velocity ub (INFLOW cells). Each column comes from one dual-number evaluation.
void cell_vjp(const Oracle& o, long n, const double* fin, const double* uref, const double mu[27], double lam[27],
              double* dgam, double dub[3]) {
  const Lat& L = o.L;
  double ubv[3];
  inlet_velocity(o, n, ubv);
  double g = gamma_at(o, n);
  const int nparam = L.Q + 4;
  for (int p = 0; p < nparam; ++p) {
    Dual f[27], fs[27], urep[3], ub[3];
    for (int i = 0; i < L.Q; ++i) f[i] = Dual(fin[i], (p == i) ? 1.0 : 0.0);
    Dual gam(g, p == L.Q ? 1.0 : 0.0);
    for (int a = 0; a < 3; ++a) ub[a] = Dual(ubv[a], p == L.Q + 1 + a ? 1.0 : 0.0);
    collide_cell<Dual>(o, n, f, gam, ub, uref, fs, urep, nullptr);
    double s = 0.0;
    for (int i = 0; i < L.Q; ++i) s += mu[i] * fs[i].d;
    if (p < L.Q) lam[p] = s;
    else if (p == L.Q) *dgam = s;
    else dub[p - L.Q - 1] = s;
  }
}

void cell_jvp(const Oracle& o, long n, const double* fin, const double* uref, const double* vf, double vg,
              const double vub[3], double out[27]) {
  const Lat& L = o.L;
  double ubv[3];
  inlet_velocity(o, n, ubv);
  Dual f[27], fs[27], urep[3], ub[3];
  for (int i = 0; i < L.Q; ++i) f[i] = Dual(fin[i], vf[i]);
  Dual gam(gamma_at(o, n), vg);
  for (int a = 0; a < 3; ++a) ub[a] = Dual(ubv[a], vub[a]);
  collide_cell<Dual>(o, n, f, gam, ub, uref, fs, urep, nullptr);
  for (int i = 0; i < L.Q; ++i) out[i] = fs[i].d;
}

}  // namespace

// =================================================================================================
// C interface for the Python test harness (ctypes).
extern "C" {

const char* orc_last_error() { return g_err.c_str(); }

void* orc_create(int q, int nx, int ny, int nz, double tau, double cs) {
  if ((q != 19 && q != 27) || nx < 1 || ny < 1 || nz < 1 || !(tau > 0.5) || cs < 0.0) {
    g_err = "orc_create: invalid arguments";
    return nullptr;
  }
  Oracle* o = new Oracle();
  o->L = make_lattice(q);
  o->nx = nx; o->ny = ny; o->nz = nz;
  o->N = long(nx) * ny * nz;
  o->tau0 = tau; o->cs = cs;
  o->mask.assign(o->N, M_FLUID);
  classify(*o);
  o->F.assign(long(q) * o->N, 0.0);
  o->P = o->F; o->Fn = o->F;
  for (int i = 0; i < q; ++i)
    for (long n = 0; n < o->N; ++n) o->F[long(i) * o->N + n] = o->L.w[i];
  init_refs(*o);
  return o;
}

void orc_destroy(void* h) { delete static_cast<Oracle*>(h); }

int orc_lattice(int q, int* c /*3q*/, double* w, int* opp, int* W, int* Wden) {
  if (q != 19 && q != 27) return 1;
  Lat L = make_lattice(q);
  for (int i = 0; i < q; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
    w[i] = L.w[i]; opp[i] = L.opp[i]; W[i] = L.W[i];
  }
  *Wden = L.Wden;
  return 0;
}

int orc_set_faces(void* h, const int* kinds) {
  Oracle& o = *static_cast<Oracle*>(h);
  for (int f = 0; f < 6; ++f) {
    if (kinds[f] < 0 || kinds[f] > 3) { g_err = "bad face kind"; return 1; }
  }
  for (int a = 0; a < 3; ++a)
    if ((kinds[2 * a] == F_PERIODIC) != (kinds[2 * a + 1] == F_PERIODIC)) { g_err = "periodic faces must pair"; return 1; }
  for (int f = 0; f < 6; ++f) o.face[f] = kinds[f];
  classify(o);
  return 0;
}

int orc_set_geometry(void* h, const uint8_t* mask, const double* ywall) {
  Oracle& o = *static_cast<Oracle*>(h);
  for (long n = 0; n < o.N; ++n)
    if (!(mask[n] == M_FLUID || mask[n] == M_SOLID || mask[n] == M_INFLOW || mask[n] == M_OUTFLOW)) {
      g_err = "invalid mask code"; return 1;
    }
  o.mask.assign(mask, mask + o.N);
  if (ywall) o.ywall.assign(ywall, ywall + o.N); else o.ywall.clear();
  classify(o);
  return 0;
}

void orc_set_force(void* h, double fx, double fy, double fz) {
  Oracle& o = *static_cast<Oracle*>(h);
  o.force[0] = fx; o.force[1] = fy; o.force[2] = fz;
}
void orc_set_inflow(void* h, const double* uin) {
  Oracle& o = *static_cast<Oracle*>(h);
  o.uin.assign(uin, uin + 3L * o.ny * o.nz);
  vm_reset(o);
}

// Vortex-method inlet: n vortices per step (0: off), vortex size sigma (cells), turbulence intensity
// I, random seed. The inlet field restarts from the mean profile.
int orc_set_vortex_inlet(void* h, int n, double sigma, double I, unsigned long long seed) {
  Oracle& o = *static_cast<Oracle*>(h);
  if (n < 0 || !(sigma > 0.0) || !(I >= 0.0)) { g_err = "bad vortex inlet parameters"; return 1; }
  o.vm_n = n; o.vm_sigma = sigma; o.vm_I = I; o.vm_seed = seed;
  vm_reset(o);
  return 0;
}
// Vortices of step t (3 values each: y, z, Gamma).
void orc_vm_vortices(void* h, long long t, double* out) {
  Oracle& o = *static_cast<Oracle*>(h);
  std::vector<Vortex> v = vm_vortices(o, long(t));
  for (size_t i = 0; i < v.size(); ++i) { out[3 * i] = v[i].y; out[3 * i + 1] = v[i].z; out[3 * i + 2] = v[i].gamma; }
}
// In-plane velocity of the given vortices (3 values each) at plane position (y, z).
void orc_vm_field(int n, const double* vort, double sigma, double y, double z, double* out2) {
  std::vector<Vortex> v(n);
  for (int i = 0; i < n; ++i) v[i] = {vort[3 * i], vort[3 * i + 1], vort[3 * i + 2]};
  vm_field(v, sigma, y, z, out2[0], out2[1]);
}
// Inlet velocity of the last step (3 * ny * nz, component-major).
void orc_inflow_field(void* h, double* out) {
  Oracle& o = *static_cast<Oracle*>(h);
  std::memcpy(out, o.uin_cur.data(), sizeof(double) * o.uin_cur.size());
}
unsigned long long orc_splitmix64(unsigned long long z) { return splitmix64_out(z); }
double orc_vm_uniform(unsigned long long seed, unsigned long long counter) { return vm_uniform(seed, counter); }
void orc_set_outflow(void* h, double rho) { static_cast<Oracle*>(h)->rho_out = rho; }
int orc_set_fringe(void* h, int L, double smax, double p, int x0) {
  Oracle* o = static_cast<Oracle*>(h);
  // L may exceed nx: a crop of a larger domain keeps the domain's layer (first plane x0)
  if (L < 0 || !(smax >= 0.0 && smax <= 1.0) || !(p >= 0.0)) {
    g_err = "fringe: need L >= 0, 0 <= s_max <= 1, p >= 0";
    return 1;
  }
  o->fr_L = L;
  o->fr_x0 = x0;
  o->fr_smax = smax;
  o->fr_p = p;
  return 0;
}
double orc_fringe_strength(void* h, int x) { return fringe_strength(*static_cast<Oracle*>(h), x); }
void orc_set_porosity(void* h, const double* g) {
  Oracle& o = *static_cast<Oracle*>(h);
  if (g) o.gamma.assign(g, g + o.N); else o.gamma.clear();
}

// Forchheimer permeability (Sec. 2.1): K = mu Q / (A (dP/L - rho Q^2 / (K_beta A^2))); K_beta = inf
// drops the inertial term (Darcy). Returns NaN when the bracket is not positive.
double orc_forchheimer_k(double mu, double Q, double A, double L, double dP, double rho, double Kbeta) {
  const double inertial = std::isinf(Kbeta) ? 0.0 : rho / Kbeta * Q * Q / (A * A);
  const double br = dP / L - inertial;
  if (!(br > 0.0)) return NAN;
  return mu * Q / (A * br);
}

// Porosity from the permeability K of every cell (lattice units, K = dx^2-scaled; +inf = fluid):
// the lattice porosity of Eq. lattice_porosity, d = 1 - dx^2 nu tau / K with dx = 1, nu = (tau - 1/2)/3
// the molecular viscosity and tau the molecular relaxation time, read as the fluid fraction
// gamma = d (gamma = 1 for K = inf, 0 for K <= 0 or NaN) clamped to [0, 1].
void orc_set_permeability(void* h, const double* K) {
  Oracle& o = *static_cast<Oracle*>(h);
  const double nu = CS2 * (o.tau0 - 0.5);
  o.gamma.assign(o.N, 1.0);
  for (long n = 0; n < o.N; ++n) {
    // K = +inf: fluid; K <= 0 or NaN carries no permeability and is read as impermeable
    double g = (std::isinf(K[n]) && K[n] > 0.0) ? 1.0 : (K[n] > 0.0 ? 1.0 - nu * o.tau0 / K[n] : 0.0);
    o.gamma[n] = std::min(1.0, std::max(0.0, g));
  }
}
void orc_get_porosity(void* h, double* g) {
  Oracle& o = *static_cast<Oracle*>(h);
  for (long n = 0; n < o.N; ++n) g[n] = o.gamma.empty() ? 1.0 : o.gamma[n];
}
void orc_set_wall_model(void* h, int on, double kappa, double E) {
  Oracle& o = *static_cast<Oracle*>(h);
  o.wm = on != 0; o.kappa = kappa; o.E = E;
}
void orc_set_storage(void* h, int mode) { static_cast<Oracle*>(h)->storage = mode; }

// Collision model: 0 BGK, 1 hybrid recursive regularised with hybridisation factor sigma in [0, 1].
int orc_set_collision(void* h, int model, double sigma) {
  Oracle& o = *static_cast<Oracle*>(h);
  if ((model != 0 && model != 1) || !(sigma >= 0.0 && sigma <= 1.0)) { g_err = "bad collision model"; return 1; }
  o.model = model;
  o.sigma = sigma;
  return 0;
}
int orc_get_collision(void* h, double* sigma) {
  Oracle& o = *static_cast<Oracle*>(h);
  *sigma = o.sigma;
  return o.model;
}

// Third-order term of every population for the symmetric tensor a (27 values, a[(a*3+b)*3+c]).
int orc_third_order(int q, const double* a27, double* out) {
  if (q != 19 && q != 27) return 1;
  Lat L = make_lattice(q);
  double a[3][3][3];
  for (int i = 0; i < 27; ++i) a[i / 9][(i / 3) % 3][i % 3] = a27[i];
  for (int i = 0; i < q; ++i) out[i] = third_term(L, i, a);
  return 0;
}
// Third-order equilibrium of every population.
int orc_feq3(int q, double rho, const double* u, double* out) {
  if (q != 19 && q != 27) return 1;
  Lat L = make_lattice(q);
  for (int i = 0; i < q; ++i) out[i] = feq3(L, i, rho, u);
  return 0;
}
// One HRR update of a cell from its density, equilibrium velocity ueq, expansion velocity uh,
// relaxation time and second-order coefficient A2 (9 values, row-major).
int orc_collide_hrr(int q, double rho, const double* ueq, const double* uh, double tau, const double* A2, double* out) {
  if (q != 19 && q != 27) return 1;
  Lat L = make_lattice(q);
  double A[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) A[a][b] = A2[3 * a + b];
  collide_hrr(L, rho, ueq, uh, tau, A, out);
  return 0;
}
// Finite-difference strain of cell n from the stored velocity field (9 values, row-major).
void orc_strain_fd(void* h, long long n, double* S9) {
  Oracle& o = *static_cast<Oracle*>(h);
  double S[3][3];
  strain_fd(o, long(n), S);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) S9[3 * a + b] = S[a][b];
}
// Velocity field of the last step (3N, component-major) as the HRR strain reads it; set_velocity_field
// replaces it (tests of the finite differences).
void orc_get_velocity_field(void* h, double* u) {
  Oracle& o = *static_cast<Oracle*>(h);
  std::memcpy(u, o.uvel_prev.data(), sizeof(double) * 3 * o.N);
}
void orc_set_velocity_field(void* h, const double* u) {
  Oracle& o = *static_cast<Oracle*>(h);
  o.uvel_prev.assign(u, u + 3 * o.N);
  o.uvel_cur = o.uvel_prev;
}

// f_i = f^eq_i(rho, u); rho (N), u (3N, component-major). Then the reference buffer is filled with
// the reported velocity of this state.
void orc_init_equilibrium(void* h, const double* rho, const double* u) {
  Oracle& o = *static_cast<Oracle*>(h);
  for (long n = 0; n < o.N; ++n) {
    double uu[3] = {u[n], u[o.N + n], u[2 * o.N + n]};
    for (int i = 0; i < o.L.Q; ++i)
      o.F[long(i) * o.N + n] = (o.kind[n] == K_SOLID) ? 0.0 : feq(o.L, i, rho[n], uu);
  }
  store_round(o, o.F);
  init_refs(o);
  o.t = 0;
}

void orc_set_populations(void* h, const double* f) {
  Oracle& o = *static_cast<Oracle*>(h);
  o.F.assign(f, f + long(o.L.Q) * o.N);
  init_refs(o);
}
void orc_get_populations(void* h, double* f) {
  Oracle& o = *static_cast<Oracle*>(h);
  std::memcpy(f, o.F.data(), sizeof(double) * o.F.size());
}
void orc_get_refbuf(void* h, double* u /*3N*/) {
  Oracle& o = *static_cast<Oracle*>(h);
  std::memcpy(u, o.uref_prev.data(), sizeof(double) * 3 * o.N);
}

void orc_step(void* h, int n) {
  Oracle& o = *static_cast<Oracle*>(h);
  for (int k = 0; k < n; ++k) step_once(o);
}

// Slab sub-domain: the first lo and last hi z-planes are ghost planes (0 or 2 each).
int orc_set_ghost(void* h, int lo, int hi) {
  Oracle& o = *static_cast<Oracle*>(h);
  if (!(lo == 0 || lo == 2) || !(hi == 0 || hi == 2) || lo + hi >= o.nz) {
    g_err = "ghost planes: 0 or 2 per side, fewer than nz in total";
    return 1;
  }
  o.gh_lo = lo;
  o.gh_hi = hi;
  return 0;
}
void orc_step_collide(void* h) { step_collide(*static_cast<Oracle*>(h)); }
void orc_step_stream(void* h) { step_stream(*static_cast<Oracle*>(h)); }
long long orc_halo_count(void* h, int side, int list) {
  return (long long)halo_list(*static_cast<Oracle*>(h), side, list).size();
}
void orc_halo_list(void* h, int side, int list, long long* out) {
  const std::vector<long> v = halo_list(*static_cast<Oracle*>(h), side, list);
  for (size_t k = 0; k < v.size(); ++k) out[k] = v[k];
}
// After the collide phase: list 0 packs the leaving post-collision populations, list 2 the
// reference velocities of this step; unpack of list 1 / list 3 stores the neighbour's into the ghost
// plane (populations into P, velocities into the reference buffer read by the next step).
void orc_halo_pack(void* h, int side, int list, double* buf) {
  Oracle& o = *static_cast<Oracle*>(h);
  const long nxy = long(o.nx) * o.ny;
  const int zr = side == 0 ? o.gh_lo : o.nz - o.gh_hi - 1;
  const std::vector<long> v = halo_list(o, side, list);
  for (size_t k = 0; k < v.size(); ++k) {
    if (list == 0) {
      const long p = v[k] / nxy, pos = v[k] % nxy;
      buf[k] = o.P[long(o.L.opp[p]) * o.N + pos + nxy * zr];
    } else {
      for (int a = 0; a < 3; ++a) buf[3 * k + a] = o.uref_cur[3 * (v[k] + nxy * zr) + a];
    }
  }
}
void orc_halo_unpack(void* h, int side, int list, const double* buf) {
  Oracle& o = *static_cast<Oracle*>(h);
  const long nxy = long(o.nx) * o.ny;
  const int zg = side == 0 ? o.gh_lo - 1 : o.nz - o.gh_hi;
  const std::vector<long> v = halo_list(o, side, list);
  for (size_t k = 0; k < v.size(); ++k) {
    if (list == 1) {
      const long p = v[k] / nxy, pos = v[k] % nxy;
      o.P[long(o.L.opp[p]) * o.N + pos + nxy * zg] = buf[k];
    } else {
      for (int a = 0; a < 3; ++a) o.uref_cur[3 * (v[k] + nxy * zg) + a] = buf[3 * k + a];
    }
  }
}

void orc_moments(void* h, double* rho, double* u) {
  Oracle& o = *static_cast<Oracle*>(h);
  moments_of(o, o.F, rho, u);
}

// mass = sum rho, mom = sum rho u (reported velocity) over non-solid cells.
void orc_reduce(void* h, double* mass, double* mom) {
  Oracle& o = *static_cast<Oracle*>(h);
  std::vector<double> rho(o.N), u(3 * o.N);
  moments_of(o, o.F, rho.data(), u.data());
  double m = 0, p[3] = {0, 0, 0};
  for (long n = 0; n < o.N; ++n) {
    if (o.kind[n] == K_SOLID || is_ghost(o, n)) continue;
    m += rho[n];
    for (int a = 0; a < 3; ++a) p[a] += rho[n] * u[a * o.N + n];
  }
  *mass = m;
  for (int a = 0; a < 3; ++a) mom[a] = p[a];
}

// Classification outputs: kind (N), isref (N), integer normal sums (3N), ref cell (N, -1 none).
void orc_classification(void* h, uint8_t* kind, uint8_t* isref, int* nsum, long long* ref) {
  Oracle& o = *static_cast<Oracle*>(h);
  for (long n = 0; n < o.N; ++n) {
    kind[n] = o.kind[n]; isref[n] = o.isref[n]; ref[n] = o.refcell[n];
    for (int a = 0; a < 3; ++a) nsum[3 * n + a] = o.nsum[3 * n + a];
  }
}

// Source map: for each non-solid cell n and direction i, src_dir[i*N+n] = j and src_cell[i*N+n] = m
// with f_i(n, t+1) = f*_j(m, t). Solid cells get -1.
void orc_source_map(void* h, int* src_dir, long long* src_cell) {
  Oracle& o = *static_cast<Oracle*>(h);
  for (int i = 0; i < o.L.Q; ++i)
    for (long n = 0; n < o.N; ++n) {
      long k = long(i) * o.N + n;
      if (o.kind[n] == K_SOLID) { src_dir[k] = -1; src_cell[k] = -1; continue; }
      int j; long m;
      source(o, n, i, j, m);
      src_dir[k] = j; src_cell[k] = m;
    }
}

// Scalar pieces for the pins.
double orc_spalding_yplus(double up, double kappa, double E) { return spalding_yplus(up, kappa, E); }
double orc_spalding_dyplus(double up, double kappa, double E) { return spalding_dyplus(up, kappa, E); }
double orc_solve_uplus_re(double Re, double kappa, double E, int* it) { return solve_uplus_from_re(Re, kappa, E, it); }
double orc_solve_uplus_yplus(double yp, double kappa, double E, int* it) { return solve_uplus_from_yplus(yp, kappa, E, it); }
double orc_tau_smagorinsky(double tau0, double cs, const double* Pi9, double rho) {
  double Pi[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Pi[a][b] = Pi9[3 * a + b];
  return tau_smagorinsky(tau0, cs, Pi, rho);
}
void orc_feq(int q, double rho, const double* u, double* out) {
  Lat L = make_lattice(q);
  for (int i = 0; i < q; ++i) out[i] = feq(L, i, rho, u);
}
// Boundary reconstruction on one cell's populations (kind 3 velocity inlet, 4 pressure outlet).
void orc_bc(int q, int kind, double* f, const double* ub, double rho_out) {
  Lat L = make_lattice(q);
  if (kind == 3) bc_velocity(L, f, ub);
  else bc_pressure(L, f, rho_out);
}
// Wall-model state of one WALL cell from the current reference buffer (for pins).
int orc_wall_state(void* h, long long n, double* uB, double* dudn) {
  Oracle& o = *static_cast<Oracle*>(h);
  if (n < 0 || n >= o.N || o.kind[n] != K_WALL) return 1;
  WallState ws = wall_state(o, n, o.uref_prev.data());
  for (int a = 0; a < 3; ++a) uB[a] = ws.uB[a];
  *dudn = ws.dudn;
  return 0;
}
uint16_t orc_f16_encode(double x) { return f16_encode(x); }
double orc_f16_decode(uint16_t b) { return f16_decode(b); }
uint16_t orc_bf16_encode(double x) { return bf16_encode(x); }
double orc_bf16_decode(uint16_t b) { return bf16_decode(b); }

// ---- differentiation -----------------------------------------------------------------------------
// Forward-mode derivative of one step at the current state: out = dS_{t+1}/dS_t vf
// + dS_{t+1}/dgamma vg + dS_{t+1}/du_in vu. The state is not advanced.
void orc_jvp_step(void* h, const double* vf, const double* vg, const double* vu, double* out) {
  Oracle& o = *static_cast<Oracle*>(h);
  const Lat& L = o.L;
  std::vector<double> dP(long(L.Q) * o.N, 0.0);
  long pl = long(o.ny) * o.nz;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < o.N; ++n) {
    if (o.kind[n] == K_SOLID) continue;
    double f[27], v[27], d[27];
    for (int i = 0; i < L.Q; ++i) { f[i] = o.F[long(i) * o.N + n]; v[i] = vf[long(i) * o.N + n]; }
    int x, y, z;
    coords(o, n, x, y, z);
    double vub[3] = {0, 0, 0};
    if (vu)
      for (int a = 0; a < 3; ++a) vub[a] = vu[a * pl + y + long(o.ny) * z];
    cell_jvp(o, n, f, o.uref_prev.data(), v, vg ? vg[n] : 0.0, vub, d);
    for (int i = 0; i < L.Q; ++i) dP[long(i) * o.N + n] = d[i];
  }
  for (long n = 0; n < o.N; ++n)
    for (int i = 0; i < L.Q; ++i) {
      long k = long(i) * o.N + n;
      if (o.kind[n] == K_SOLID) { out[k] = 0.0; continue; }
      int j; long m;
      source(o, n, i, j, m);
      out[k] = dP[long(j) * o.N + m];
    }
}

// Transpose of the step derivative at the current state: given w (sensitivity of S_{t+1}), return
// out_f = (dS_{t+1}/dS_t)^T w, out_g += (dS_{t+1}/dgamma)^T w, out_u += (dS_{t+1}/du_in)^T w.
static void vjp_at(Oracle& o, const std::vector<double>& Fst, const double* uref, const double* w, double* out_f,
                   double* out_g, double* out_u) {
  const Lat& L = o.L;
  std::vector<double> mu(long(L.Q) * o.N, 0.0);
  for (long n = 0; n < o.N; ++n) {
    if (o.kind[n] == K_SOLID) continue;
    for (int i = 0; i < L.Q; ++i) {
      int j; long m;
      source(o, n, i, j, m);
      mu[long(j) * o.N + m] += w[long(i) * o.N + n];
    }
  }
  long pl = long(o.ny) * o.nz;
  std::vector<double> dub(3 * o.N, 0.0);
#pragma omp parallel for schedule(static)
  for (long n = 0; n < o.N; ++n) {
    if (o.kind[n] == K_SOLID) {
      for (int i = 0; i < L.Q; ++i) out_f[long(i) * o.N + n] = 0.0;
      continue;
    }
    double f[27], m[27], lam[27], dg = 0.0, du[3] = {0, 0, 0};
    for (int i = 0; i < L.Q; ++i) { f[i] = Fst[long(i) * o.N + n]; m[i] = mu[long(i) * o.N + n]; }
    cell_vjp(o, n, f, uref, m, lam, &dg, du);
    for (int i = 0; i < L.Q; ++i) out_f[long(i) * o.N + n] = lam[i];
    if (out_g) out_g[n] += dg;
    for (int a = 0; a < 3; ++a) dub[3 * n + a] = du[a];
  }
  if (out_u)
    for (long n = 0; n < o.N; ++n) {
      if (o.kind[n] != K_INFLOW) continue;
      int x, y, z;
      coords(o, n, x, y, z);
      for (int a = 0; a < 3; ++a) out_u[a * pl + y + long(o.ny) * z] += dub[3 * n + a];
    }
}

void orc_vjp_step(void* h, const double* w, double* out_f, double* out_g, double* out_u) {
  Oracle& o = *static_cast<Oracle*>(h);
  vjp_at(o, o.F, o.uref_prev.data(), w, out_f, out_g, out_u);
}

// Pressure-drop objective (reading of the differentiation workload): over the last W of T steps,
// J = (1/W) sum_t cs^2 (<rho>_{x=xa} - <rho>_{x=xb}), plane means over non-solid cells, rho of the
// pre-collision state S_t after step t. Runs T steps from the current state, storing every state
// for the reverse sweep. The planes must not hold INFLOW/OUTFLOW cells.
int orc_objective_run(void* h, int T, int W, int xa, int xb, double* J) {
  Oracle& o = *static_cast<Oracle*>(h);
  if (T < 1 || W < 1 || W > T || xa < 0 || xa >= o.nx || xb < 0 || xb >= o.nx) { g_err = "bad objective args"; return 1; }
  if (o.model != 0) { g_err = "the adjoint is defined for the BGK collision only"; return 1; }
  if (o.vm_n != 0) { g_err = "the adjoint is defined for a steady inlet only"; return 1; }
  const Lat& L = o.L;
  o.dJdS_w.assign(o.N, 0.0);
  long na = 0, nb = 0;
  for (long n = 0; n < o.N; ++n) {
    int x, y, z;
    coords(o, n, x, y, z);
    if (o.kind[n] == K_SOLID) continue;
    if ((x == xa || x == xb) && (o.kind[n] == K_INFLOW || o.kind[n] == K_OUTFLOW)) { g_err = "objective plane holds boundary cells"; return 1; }
    if (x == xa) ++na;
    if (x == xb) ++nb;
  }
  for (long n = 0; n < o.N; ++n) {
    int x, y, z;
    coords(o, n, x, y, z);
    if (o.kind[n] == K_SOLID) continue;
    if (x == xa) o.dJdS_w[n] += CS2 / (double(W) * na);
    if (x == xb) o.dJdS_w[n] -= CS2 / (double(W) * nb);
  }
  o.hist.clear(); o.href.clear();
  double acc = 0.0;
  for (int t = 0; t < T; ++t) {
    o.hist.push_back(o.F);
    o.href.push_back(o.uref_prev);
    step_once(o);
    if (t + 1 > T - W) {
      for (long n = 0; n < o.N; ++n) {
        if (o.dJdS_w[n] == 0.0) continue;
        double r = 0.0;
        for (int i = 0; i < L.Q; ++i) r += o.F[long(i) * o.N + n];
        acc += o.dJdS_w[n] * r;
      }
    }
  }
  o.T_run = T; o.W_run = W;
  *J = acc;
  return 0;
}

// Reverse sweep after orc_objective_run: dJ/dgamma (N) and dJ/du_in (3 ny nz), both accumulated
// over all steps. lambda_T = dJ/dS_T; lambda_t = M_t^T lambda_{t+1} + dJ/dS_t.
int orc_adjoint(void* h, double* dJdg, double* dJdu) {
  Oracle& o = *static_cast<Oracle*>(h);
  if (o.hist.empty()) { g_err = "no stored run"; return 1; }
  const Lat& L = o.L;
  long T = o.T_run, W = o.W_run;
  std::fill(dJdg, dJdg + o.N, 0.0);
  std::fill(dJdu, dJdu + 3L * o.ny * o.nz, 0.0);
  std::vector<double> lam(long(L.Q) * o.N, 0.0), prev(long(L.Q) * o.N, 0.0);
  auto add_dJ = [&](std::vector<double>& l) {
    for (long n = 0; n < o.N; ++n)
      if (o.dJdS_w[n] != 0.0)
        for (int i = 0; i < L.Q; ++i) l[long(i) * o.N + n] += o.dJdS_w[n];
  };
  add_dJ(lam);  // t = T is always in the window
  for (long t = T - 1; t >= 0; --t) {
    vjp_at(o, o.hist[t], o.href[t].data(), lam.data(), prev.data(), dJdg, dJdu);
    std::swap(lam, prev);
    if (t > T - W) add_dJ(lam);
  }
  return 0;
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n);
#else
  (void)n;
#endif
}
int orc_get_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
