// soliton_oracle.cpp -- plain FP64 CPU restatement of the soliton relaxation method.
//
// TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
// cpu_baseline / reference leg load this library. The product (the CUDA library
// under paper_2603_24370_gb300/csrc) never includes, links or calls it, and the
// two share no code: no header, no helper, no constant table.
//
// Equation numbering follows the order of appearance in the paper (its equations
// are unnumbered in print):
//   Eq. 1  4th-order first-derivative stencil            (Sec. 3.1)
//   Eq. 2  4th-order second-derivative stencil           (Sec. 3.1)
//   Eq. 3  arrested Newton flow  phi'' = -grad E_h       (Sec. 3.2)
//   Eq. 4  arrest test  E_h[phi^{n+1}] > E_h[phi^n]      (Sec. 3.2)
//   Eq. 5  chiral-magnet energy functional               (Sec. 4.2)
//   Table 1  energy functionals (Abelian Higgs and Baby Skyrme rows)  (Sec. 2.3)
//
// Readings of points the paper leaves open (each is listed with its reason in the
// design notes of the repository):
//   * The array is nx x ny sites including a halo of width 2 (Sec. 3.1). The halo
//     keeps the initial values for ever (Dirichlet); only interior sites
//     I = [2, nx-3] x [2, ny-3] are updated.
//   * Coordinates x_i = (i - (nx-1)/2) dx, y_j = (j - (ny-1)/2) dy; i runs along x
//     and is the fastest index; planes are stored [C][ny][nx].
//   * E_h = dx dy sum_I e, with e evaluated with Eq. 1 only.
//   * The force G that drives Eq. 3 is the continuum Euler-Lagrange expression with
//     Eq. 1 / Eq. 2 derivatives (and Eq. 1 in x composed with Eq. 1 in y for the
//     mixed derivative); it is the density-form residual, so the flow has unit wave
//     speed and dt = C min(dx, dy) with C = 0.5 (Sec. 3.1).
//   * The exact gradient of E_h (adjoint of Eq. 1) is provided separately, only for
//     the tests that pin G.
//   * Chiral magnet: interfacial DMI vectors d_1 = e_3 x e_1, d_2 = e_3 x e_2 by
//     default, no demagnetising term; the unit-length constraint is enforced by
//     normalising every RK stage input and the new field, tangent-projecting the
//     force and the new velocity (Sec. 3.2, projection paragraph).
//   * Baby Skyrme (Table 1): the Skyrme term's double sum over i, j is
//     kappa^2/2 |d_1 m x d_2 m|^2; potential mu^2 (1 - m_3) + nu^2/2 m_1^2; the unit
//     vector is projected exactly as the chiral magnet's.
//   * Rotating BEC (Table 1; the BEC section): dimensionless (hbar = m = omega = 1),
//     in the grand-canonical form at chemical potential mu: the functional minimised is
//     E - mu N, which fixes the atom number N at the minimum; Re(psi* L_z psi) is the
//     rotation density (its imaginary part is a total derivative).
//   * s+id superconductor (Table 1): gradient tensor gamma^{ss}_{jk} = gamma^{dd}_{jk} =
//     delta_jk and gamma^{sd}_{jk} = gamma^{ds}_{jk} = nu diag(1, -1)_{jk} (the
//     d_{x^2-y^2} mixed gradient), unit charge D = d - i A, components
//     (Re, Im Delta_s, Re, Im Delta_d, A_1, A_2). params = {a1, a2, b1, b2, b3, b4, nu}.
//   * Demagnetisation (Eq. 6, the chiral magnet with demag, theory 6): with
//     psi = phi / (mu_0 M_s) the Poisson equation reads lap psi = div n (in-plane n),
//     discretised as L psi = rho on a Dirichlet box B containing I: rho the Eq. 1
//     divergence of (n_1, n_2) on I and zero on the rest of B, L the 5-point Laplacian,
//     psi = 0 on the nodes just outside B (standing in for the far field). Along each
//     axis B has the N' >= N sites with N' + 1 the first size free of prime factors
//     above 7, floor((N' - N) / 2) of the extra sites below I and the rest above, so
//     the sine transform has an FFT-friendly length (B = I when N + 1 already is).
//     Only psi on I enters: the stored potential is psi on I and zero on the halo.
//     Energy E_ms = 1/(2 mu_0) int |grad phi|^2 = -mu_d/2 int psi rho with
//     mu_d = mu_0 M_s^2, discretised as -mu_d/2 dx dy sum_I psi rho, whose exact lattice
//     gradient is mu_d dx dy (Eq. 1 gradient of psi) because L is symmetric and Eq. 1
//     antisymmetric: the force is G_cm + mu_d (d_1 psi, d_2 psi, 0), then projected.
//     Within a flow step psi is solved once, for the step's starting field, and held
//     through the RK stages; every energy uses the psi of its own field.
//     params = {J, D, K, h, dmi_type, mu_d}.
//   * Arrest compares potential energies with a strict '>' (Eq. 4).
//   * Convergence measure: max over I and components of |dx dy G|.
#include <cmath>
#include <cstdint>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <cstring>
#include <vector>

namespace {

const double PI = 3.14159265358979323846;

enum { TH_ABELIAN_HIGGS = 1, TH_CHIRAL_MAGNET = 2, TH_BABY_SKYRME = 3, TH_BEC = 4, TH_SID = 5,
       TH_CM_DEMAG = 6, TH_HARMONIC_TEST = 99 };

// Theories whose field is a unit 3-vector (normalised after every update).
bool unit_vector(int theory) {
  return theory == TH_CHIRAL_MAGNET || theory == TH_BABY_SKYRME || theory == TH_CM_DEMAG;
}

struct Grid {
  int nx, ny;
  double dx, dy;
  size_t plane() const { return (size_t)nx * ny; }
  bool interior(int i, int j) const { return i >= 2 && i <= nx - 3 && j >= 2 && j <= ny - 3; }
};

int ncomp(int theory) {
  switch (theory) {
    case TH_ABELIAN_HIGGS: return 4;   // psi_1, psi_2, A_1, A_2 (Table 1)
    case TH_CHIRAL_MAGNET: return 3;   // n_1, n_2, n_3 (Eq. 5)
    case TH_BABY_SKYRME: return 3;     // m_1, m_2, m_3 (Table 1)
    case TH_BEC: return 2;             // Re psi, Im psi (Table 1)
    case TH_SID: return 6;             // Delta_s, Delta_d (Re, Im), A_1, A_2 (Table 1)
    case TH_CM_DEMAG: return 3;        // n (Eq. 5 with the magnetostatic term)
    case TH_HARMONIC_TEST: return 1;   // scalar test field
    default: return 0;
  }
}

// Neumaier compensated sum, fixed (row-major) order.
struct Neumaier {
  double s = 0.0, c = 0.0;
  void add(double x) {
    double t = s + x;
    if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

// ---------------------------------------------------------------- stencils
// Eq. 1 (Sec. 3.1): d_x phi_{i,j} ~ (-phi_{i+2} + 8 phi_{i+1} - 8 phi_{i-1} + phi_{i-2}) / (12 dx)
double d1x(const double* p, const Grid& g, int i, int j) {
  const double* r = p + (size_t)j * g.nx;
  return (-r[i + 2] + 8.0 * r[i + 1] - 8.0 * r[i - 1] + r[i - 2]) / (12.0 * g.dx);
}
// Eq. 1, "analogous expression in the y direction".
double d1y(const double* p, const Grid& g, int i, int j) {
  const size_t n = g.nx;
  return (-p[(j + 2) * n + i] + 8.0 * p[(j + 1) * n + i] - 8.0 * p[(j - 1) * n + i] + p[(j - 2) * n + i]) /
         (12.0 * g.dy);
}
// Eq. 2 (Sec. 3.1): d_x^2 phi ~ (-phi_{i+2} + 16 phi_{i+1} - 30 phi_i + 16 phi_{i-1} - phi_{i-2}) / (12 dx^2)
double d2x(const double* p, const Grid& g, int i, int j) {
  const double* r = p + (size_t)j * g.nx;
  return (-r[i + 2] + 16.0 * r[i + 1] - 30.0 * r[i] + 16.0 * r[i - 1] - r[i - 2]) / (12.0 * g.dx * g.dx);
}
double d2y(const double* p, const Grid& g, int i, int j) {
  const size_t n = g.nx;
  return (-p[(j + 2) * n + i] + 16.0 * p[(j + 1) * n + i] - 30.0 * p[j * n + i] + 16.0 * p[(j - 1) * n + i] -
          p[(j - 2) * n + i]) /
         (12.0 * g.dy * g.dy);
}
// Mixed derivative d_x d_y: Eq. 1 along y applied to Eq. 1 along x (the paper is
// silent on mixed derivatives; this is the composition of its two stencils).
double d12(const double* p, const Grid& g, int i, int j) {
  return (-d1x(p, g, i, j + 2) + 8.0 * d1x(p, g, i, j + 1) - 8.0 * d1x(p, g, i, j - 1) + d1x(p, g, i, j - 2)) /
         (12.0 * g.dy);
}

// All derivatives of every component at one interior site, and its coordinates.
struct Site {
  double v[6], fx[6], fy[6], fxx[6], fyy[6], fxy[6];
  double x, y;
};

Site gather(const double* f, int C, const Grid& g, int i, int j, bool second) {
  Site s;
  s.x = (i - 0.5 * (g.nx - 1)) * g.dx;
  s.y = (j - 0.5 * (g.ny - 1)) * g.dy;
  for (int c = 0; c < C; ++c) {
    const double* p = f + c * g.plane();
    s.v[c] = p[(size_t)j * g.nx + i];
    s.fx[c] = d1x(p, g, i, j);
    s.fy[c] = d1y(p, g, i, j);
    if (second) {
      s.fxx[c] = d2x(p, g, i, j);
      s.fyy[c] = d2y(p, g, i, j);
      s.fxy[c] = d12(p, g, i, j);
    } else {
      s.fxx[c] = s.fyy[c] = s.fxy[c] = 0.0;
    }
  }
  return s;
}

// DMI vectors d_1, d_2 (Eq. 5). type 0: interfacial d_i = e_3 x e_i (Neel);
// type 1: bulk d_i = e_i (Bloch); type 2: d_1 = e_1, d_2 = -e_2 (D_2d, "Heusler",
// anti-skyrmions; Sec. 4.2).
void dmi_vectors(int type, double d1[3], double d2[3]) {
  for (int k = 0; k < 3; ++k) d1[k] = d2[k] = 0.0;
  if (type == 1) { d1[0] = 1.0; d2[1] = 1.0; }
  else if (type == 2) { d1[0] = 1.0; d2[1] = -1.0; }
  else { d1[1] = 1.0; d2[0] = -1.0; }  // e3 x e1 = e2, e3 x e2 = -e1
}

void cross(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}
double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// ---------------------------------------------------------------- energy densities
// Abelian Higgs (Table 1): e = 1/2 |D psi|^2 + 1/2 |curl A|^2 + lambda/8 (u^2 - |psi|^2)^2,
// with D_i psi = d_i psi - i A_i psi (unit charge). params = {lambda, u}.
double density_ah(const double* prm, const Site& s) {
  const double lam = prm[0], u = prm[1];
  const double p1 = s.v[0], p2 = s.v[1], A1 = s.v[2], A2 = s.v[3];
  // D_i psi = (d_i psi_1 + A_i psi_2) + i (d_i psi_2 - A_i psi_1)
  const double re1 = s.fx[0] + A1 * p2, im1 = s.fx[1] - A1 * p1;
  const double re2 = s.fy[0] + A2 * p2, im2 = s.fy[1] - A2 * p1;
  const double B = s.fx[3] - s.fy[2];  // d_1 A_2 - d_2 A_1
  const double w = u * u - (p1 * p1 + p2 * p2);
  return 0.5 * (re1 * re1 + im1 * im1 + re2 * re2 + im2 * im2) + 0.5 * B * B + lam / 8.0 * w * w;
}

// Chiral magnet (Eq. 5 without the demagnetising term, dimensionless):
// e = J/2 |d n|^2 + D sum_i d_i . (n x d_i n) + K (1 - n_3^2) + h (1 - n_3).
// params = {J, D, K, h, dmi_type}.
double density_cm(const double* prm, const Site& s) {
  const double J = prm[0], D = prm[1], K = prm[2], h = prm[3];
  double dv1[3], dv2[3];
  dmi_vectors((int)prm[4], dv1, dv2);
  const double n[3] = {s.v[0], s.v[1], s.v[2]};
  const double nx_[3] = {s.fx[0], s.fx[1], s.fx[2]};
  const double ny_[3] = {s.fy[0], s.fy[1], s.fy[2]};
  double c1[3], c2[3];
  cross(n, nx_, c1);
  cross(n, ny_, c2);
  const double ex = 0.5 * J * (dot3(nx_, nx_) + dot3(ny_, ny_));
  const double dmi = D * (dot3(dv1, c1) + dot3(dv2, c2));
  return ex + dmi + K * (1.0 - n[2] * n[2]) + h * (1.0 - n[2]);
}

// Baby Skyrme (Table 1): e = 1/2 |d m|^2 + kappa^2/4 sum_{i,j} |d_i m x d_j m|^2 + V(m).
// The double sum counts d_1 m x d_2 m twice and the diagonal terms vanish, so the
// Skyrme term is kappa^2/2 |d_1 m x d_2 m|^2. Potential family
// V = mu^2 (1 - m_3) + nu^2/2 m_1^2 (the standard potential at nu = 0, the easy-plane
// one at mu = 0). prm = {kappa, mu, nu}.
double density_bs(const double* prm, const Site& s) {
  const double k2 = prm[0] * prm[0], mu2 = prm[1] * prm[1], nu2 = prm[2] * prm[2];
  const double a[3] = {s.fx[0], s.fx[1], s.fx[2]}, b[3] = {s.fy[0], s.fy[1], s.fy[2]};
  double X[3];
  cross(a, b, X);
  return 0.5 * (dot3(a, a) + dot3(b, b)) + 0.5 * k2 * dot3(X, X) + mu2 * (1.0 - s.v[2]) +
         0.5 * nu2 * s.v[0] * s.v[0];
}

// Rotating trapped BEC (Table 1), dimensionless (hbar = m = omega = 1), grand canonical:
//   e = 1/2 |grad psi|^2 + 1/2 r^2 |psi|^2 + g/2 |psi|^4 - mu |psi|^2 - Omega Re(psi* L_z psi),
// L_z = -i (x d_y - y d_x); with psi = u + i v and D = x d_y - y d_x,
//   psi* L_z psi = (u D v - v D u) - i/2 D(u^2 + v^2),
// whose imaginary part integrates to zero. prm = {g, Omega, mu}.
double density_bec(const double* prm, const Site& s) {
  const double g = prm[0], Om = prm[1], mu = prm[2];
  const double u = s.v[0], v = s.v[1];
  const double Du = s.x * s.fy[0] - s.y * s.fx[0], Dv = s.x * s.fy[1] - s.y * s.fx[1];
  const double n = u * u + v * v, r2 = s.x * s.x + s.y * s.y;
  const double kin = 0.5 * (s.fx[0] * s.fx[0] + s.fy[0] * s.fy[0] + s.fx[1] * s.fx[1] + s.fy[1] * s.fy[1]);
  return kin + 0.5 * r2 * n + 0.5 * g * n * n - mu * n - Om * (u * Dv - v * Du);
}

// s+id two-band Ginzburg-Landau model (Table 1):
//   e = 1/2 gamma^{ab}_{jk} (D_j Delta_a)* D_k Delta_b + 1/2 B^2 + a1 |Ds|^2 + a2 |Dd|^2
//       + b1 |Ds|^4 + b2 |Dd|^4 + b3 |Ds|^2 |Dd|^2 + b4 (Ds^2 conj(Dd)^2 + c.c.),
// with Ds = Delta_s, Dd = Delta_d. In real components, for band a = (u_a + i w_a):
//   X_aj = Re D_j Delta_a = d_j u_a + A_j w_a,  Y_aj = Im D_j Delta_a = d_j w_a - A_j u_a,
// the gradient energy is 1/2 sum_{a,j} (X_aj^2 + Y_aj^2) + nu sum_j eta_j (X_sj X_dj + Y_sj Y_dj),
// eta = (1, -1); with p + i q = Ds conj(Dd), Ds^2 conj(Dd)^2 + c.c. = 2 (p^2 - q^2).
struct SidTerms {
  double X[2][2], Y[2][2];  // [band][direction]
  double S, Dd, p, q, B;
};
SidTerms sid_terms(const Site& s) {
  SidTerms t;
  const double A[2] = {s.v[4], s.v[5]};
  for (int a = 0; a < 2; ++a) {
    const double u = s.v[2 * a], w = s.v[2 * a + 1];
    const double du[2] = {s.fx[2 * a], s.fy[2 * a]}, dw[2] = {s.fx[2 * a + 1], s.fy[2 * a + 1]};
    for (int j = 0; j < 2; ++j) {
      t.X[a][j] = du[j] + A[j] * w;
      t.Y[a][j] = dw[j] - A[j] * u;
    }
  }
  t.S = s.v[0] * s.v[0] + s.v[1] * s.v[1];
  t.Dd = s.v[2] * s.v[2] + s.v[3] * s.v[3];
  t.p = s.v[0] * s.v[2] + s.v[1] * s.v[3];
  t.q = s.v[1] * s.v[2] - s.v[0] * s.v[3];
  t.B = s.fx[5] - s.fy[4];
  return t;
}
double density_sid(const double* prm, const Site& s) {
  const double a1 = prm[0], a2 = prm[1], b1 = prm[2], b2 = prm[3], b3 = prm[4], b4 = prm[5], nu = prm[6];
  const SidTerms t = sid_terms(s);
  double grad = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 2; ++j) grad += 0.5 * (t.X[a][j] * t.X[a][j] + t.Y[a][j] * t.Y[a][j]);
  const double eta[2] = {1.0, -1.0};
  double mix = 0.0;
  for (int j = 0; j < 2; ++j) mix += eta[j] * (t.X[0][j] * t.X[1][j] + t.Y[0][j] * t.Y[1][j]);
  const double V = a1 * t.S + a2 * t.Dd + b1 * t.S * t.S + b2 * t.Dd * t.Dd + b3 * t.S * t.Dd +
                   2.0 * b4 * (t.p * t.p - t.q * t.q);
  return grad + nu * mix + 0.5 * t.B * t.B + V;
}

// Harmonic test theory (oracle only, pins the time integrator): e = k/2 phi^2.
double density_harm(const double* prm, const Site& s) { return 0.5 * prm[0] * s.v[0] * s.v[0]; }

double density(int theory, const double* prm, const Site& s) {
  switch (theory) {
    case TH_ABELIAN_HIGGS: return density_ah(prm, s);
    case TH_CHIRAL_MAGNET: return density_cm(prm, s);
    case TH_CM_DEMAG: return density_cm(prm, s);  // local part; E_ms is added over the lattice
    case TH_BABY_SKYRME: return density_bs(prm, s);
    case TH_BEC: return density_bec(prm, s);
    case TH_SID: return density_sid(prm, s);
    default: return density_harm(prm, s);
  }
}

// ---------------------------------------------------------------- Euler-Lagrange forces
// Abelian Higgs: G = delta E / delta phi written out from Table 1:
//   G_psi = -D_i D_i psi - lambda/2 (u^2 - |psi|^2) psi
//         = -lap psi + i (div A) psi + 2 i A_i d_i psi + |A|^2 psi - lambda/2 (u^2-|psi|^2) psi
//   G_A1  =  d_2 B - Im(conj(psi) D_1 psi),   G_A2 = -d_1 B - Im(conj(psi) D_2 psi),
//   with B = d_1 A_2 - d_2 A_1 and -Im(conj(psi) D_i psi) = psi_2 d_i psi_1 - psi_1 d_i psi_2 + A_i |psi|^2.
void force_ah(const double* prm, const Site& s, double G[4]) {
  const double lam = prm[0], u = prm[1];
  const double p1 = s.v[0], p2 = s.v[1], A1 = s.v[2], A2 = s.v[3];
  const double lap1 = s.fxx[0] + s.fyy[0], lap2 = s.fxx[1] + s.fyy[1];
  const double divA = s.fx[2] + s.fy[3];
  const double AA = A1 * A1 + A2 * A2, mod2 = p1 * p1 + p2 * p2;
  const double pot = 0.5 * lam * (u * u - mod2);
  // Re and Im of 2 i A_i d_i psi:  2 i A_i (d_i psi_1 + i d_i psi_2) = -2 A_i d_i psi_2 + 2 i A_i d_i psi_1
  G[0] = -lap1 - 2.0 * (A1 * s.fx[1] + A2 * s.fy[1]) - divA * p2 + AA * p1 - pot * p1;
  G[1] = -lap2 + 2.0 * (A1 * s.fx[0] + A2 * s.fy[0]) + divA * p1 + AA * p2 - pot * p2;
  const double d2B = s.fxy[3] - s.fyy[2];  // d_2 (d_1 A_2 - d_2 A_1)
  const double d1B = s.fxx[3] - s.fxy[2];  // d_1 (d_1 A_2 - d_2 A_1)
  G[2] = d2B + (p2 * s.fx[0] - p1 * s.fx[1]) + A1 * mod2;
  G[3] = -d1B + (p2 * s.fy[0] - p1 * s.fy[1]) + A2 * mod2;
}

// Chiral magnet: delta E / delta n = -J lap n - 2 D sum_i d_i x d_i n - 2 K n_3 e_3 - h e_3,
// then the tangent projection G <- G - (G . n) n that keeps |n| = 1 (Sec. 3.2). With
// demagnetisation, mu_d (d_1 psi, d_2 psi, 0) is added before the projection (psi_g:
// the Eq. 1 gradient of the magnetostatic potential at the site, else NULL).
void force_cm(const double* prm, const Site& s, double G[3], const double* psi_g = nullptr) {
  const double J = prm[0], D = prm[1], K = prm[2], h = prm[3];
  double dv1[3], dv2[3];
  dmi_vectors((int)prm[4], dv1, dv2);
  const double nx_[3] = {s.fx[0], s.fx[1], s.fx[2]};
  const double ny_[3] = {s.fy[0], s.fy[1], s.fy[2]};
  double c1[3], c2[3];
  cross(dv1, nx_, c1);
  cross(dv2, ny_, c2);
  for (int a = 0; a < 3; ++a) G[a] = -J * (s.fxx[a] + s.fyy[a]) - 2.0 * D * (c1[a] + c2[a]);
  G[2] += -2.0 * K * s.v[2] - h;
  if (psi_g) {
    G[0] += prm[5] * psi_g[0];
    G[1] += prm[5] * psi_g[1];
  }
  const double n[3] = {s.v[0], s.v[1], s.v[2]};
  const double gn = dot3(G, n);
  for (int a = 0; a < 3; ++a) G[a] -= gn * n[a];
}

// Baby Skyrme: with a = d_1 m, b = d_2 m the Skyrme term S = kappa^2/2 (|a|^2 |b|^2 - (a.b)^2)
// has dS/da = kappa^2 (|b|^2 a - (a.b) b), dS/db = kappa^2 (|a|^2 b - (a.b) a), and
//   -d_1 dS/da - d_2 dS/db = -kappa^2 [ |b|^2 m_11 + |a|^2 m_22 - 2 (a.b) m_12
//                                       + (b.m_12 - a.m_22) a + (a.m_12 - b.m_11) b ].
// G = -lap m + that + dV/dm, then G <- G - (G . m) m.
void force_bs(const double* prm, const Site& s, double G[3]) {
  const double k2 = prm[0] * prm[0], mu2 = prm[1] * prm[1], nu2 = prm[2] * prm[2];
  const double a[3] = {s.fx[0], s.fx[1], s.fx[2]}, b[3] = {s.fy[0], s.fy[1], s.fy[2]};
  const double m11[3] = {s.fxx[0], s.fxx[1], s.fxx[2]}, m22[3] = {s.fyy[0], s.fyy[1], s.fyy[2]};
  const double m12[3] = {s.fxy[0], s.fxy[1], s.fxy[2]};
  const double aa = dot3(a, a), bb = dot3(b, b), ab = dot3(a, b);
  const double ca = dot3(b, m12) - dot3(a, m22), cb = dot3(a, m12) - dot3(b, m11);
  for (int c = 0; c < 3; ++c)
    G[c] = -(m11[c] + m22[c]) - k2 * (bb * m11[c] + aa * m22[c] - 2.0 * ab * m12[c] + ca * a[c] + cb * b[c]);
  G[0] += nu2 * s.v[0];
  G[2] -= mu2;
  const double n[3] = {s.v[0], s.v[1], s.v[2]};
  const double gn = dot3(G, n);
  for (int c = 0; c < 3; ++c) G[c] -= gn * n[c];
}

// BEC: delta E / delta u = -lap u + r^2 u + 2 g |psi|^2 u - 2 mu u - 2 Omega D v,
//      delta E / delta v = -lap v + r^2 v + 2 g |psi|^2 v - 2 mu v + 2 Omega D u
// (half of it is the Gross-Pitaevskii operator minus mu: -lap/2 + r^2/2 + g|psi|^2 - Omega L_z - mu).
void force_bec(const double* prm, const Site& s, double G[2]) {
  const double g = prm[0], Om = prm[1], mu = prm[2];
  const double u = s.v[0], v = s.v[1];
  const double Du = s.x * s.fy[0] - s.y * s.fx[0], Dv = s.x * s.fy[1] - s.y * s.fx[1];
  const double w = s.x * s.x + s.y * s.y + 2.0 * g * (u * u + v * v) - 2.0 * mu;
  G[0] = -(s.fxx[0] + s.fyy[0]) + w * u - 2.0 * Om * Dv;
  G[1] = -(s.fxx[1] + s.fyy[1]) + w * v + 2.0 * Om * Du;
}

// s+id: with P_aj = X_aj + nu eta_j X_bj, Q_aj = Y_aj + nu eta_j Y_bj (b the other band),
// the conjugates of d_j u_a and d_j w_a, the Euler-Lagrange expressions are
//   G_{u_a} = -sum_j [A_j Q_aj + d_j P_aj] + dV/du_a,  G_{w_a} = sum_j [A_j P_aj - d_j Q_aj] + dV/dw_a,
//   G_{A_1} = d_2 B + sum_a (P_a1 w_a - Q_a1 u_a),  G_{A_2} = -d_1 B + sum_a (P_a2 w_a - Q_a2 u_a),
// where d_j X_aj = d_j^2 u_a + (d_j A_j) w_a + A_j d_j w_a, d_j Y_aj = d_j^2 w_a - (d_j A_j) u_a - A_j d_j u_a.
void force_sid(const double* prm, const Site& s, double G[6]) {
  const double a1 = prm[0], a2 = prm[1], b1 = prm[2], b2 = prm[3], b3 = prm[4], b4 = prm[5], nu = prm[6];
  const SidTerms t = sid_terms(s);
  const double A[2] = {s.v[4], s.v[5]}, dA[2] = {s.fx[4], s.fy[5]};
  const double eta[2] = {1.0, -1.0};
  double dX[2][2], dY[2][2];  // d_j X_aj, d_j Y_aj
  for (int a = 0; a < 2; ++a) {
    const double u = s.v[2 * a], w = s.v[2 * a + 1];
    const double du[2] = {s.fx[2 * a], s.fy[2 * a]}, dw[2] = {s.fx[2 * a + 1], s.fy[2 * a + 1]};
    const double uu[2] = {s.fxx[2 * a], s.fyy[2 * a]}, ww[2] = {s.fxx[2 * a + 1], s.fyy[2 * a + 1]};
    for (int j = 0; j < 2; ++j) {
      dX[a][j] = uu[j] + dA[j] * w + A[j] * dw[j];
      dY[a][j] = ww[j] - dA[j] * u - A[j] * du[j];
    }
  }
  // potential derivatives
  const double s1 = s.v[0], s2 = s.v[1], d1 = s.v[2], d2 = s.v[3];
  double dV[4];
  dV[0] = 2 * a1 * s1 + 4 * b1 * t.S * s1 + 2 * b3 * t.Dd * s1 + 4 * b4 * (t.p * d1 + t.q * d2);
  dV[1] = 2 * a1 * s2 + 4 * b1 * t.S * s2 + 2 * b3 * t.Dd * s2 + 4 * b4 * (t.p * d2 - t.q * d1);
  dV[2] = 2 * a2 * d1 + 4 * b2 * t.Dd * d1 + 2 * b3 * t.S * d1 + 4 * b4 * (t.p * s1 - t.q * s2);
  dV[3] = 2 * a2 * d2 + 4 * b2 * t.Dd * d2 + 2 * b3 * t.S * d2 + 4 * b4 * (t.p * s2 + t.q * s1);
  G[4] = s.fxy[5] - s.fyy[4];   //  d_2 B
  G[5] = s.fxy[4] - s.fxx[5];   // -d_1 B
  for (int a = 0; a < 2; ++a) {
    const int b = 1 - a;
    const double u = s.v[2 * a], w = s.v[2 * a + 1];
    double gu = dV[2 * a], gw = dV[2 * a + 1];
    for (int j = 0; j < 2; ++j) {
      const double P = t.X[a][j] + nu * eta[j] * t.X[b][j], Q = t.Y[a][j] + nu * eta[j] * t.Y[b][j];
      const double dP = dX[a][j] + nu * eta[j] * dX[b][j], dQ = dY[a][j] + nu * eta[j] * dY[b][j];
      gu += -A[j] * Q - dP;
      gw += A[j] * P - dQ;
      G[4 + j] += P * w - Q * u;
    }
    G[2 * a] = gu;
    G[2 * a + 1] = gw;
  }
}

void force_site(int theory, const double* prm, const Site& s, double* G) {
  switch (theory) {
    case TH_ABELIAN_HIGGS: force_ah(prm, s, G); break;
    case TH_CHIRAL_MAGNET: force_cm(prm, s, G); break;
    case TH_BABY_SKYRME: force_bs(prm, s, G); break;
    case TH_BEC: force_bec(prm, s, G); break;
    case TH_SID: force_sid(prm, s, G); break;
    default: G[0] = prm[0] * s.v[0]; break;
  }
}

// ---------------------------------------------------------------- partial derivatives of e
// d e / d phi_c and d e / d(d_i phi_c), used only by the exact gradient of E_h.
void partials(int theory, const double* prm, const Site& s, double dv[6], double dgx[6], double dgy[6]) {
  for (int c = 0; c < 6; ++c) dv[c] = dgx[c] = dgy[c] = 0.0;
  if (theory == TH_ABELIAN_HIGGS) {
    const double lam = prm[0], u = prm[1];
    const double p1 = s.v[0], p2 = s.v[1], A1 = s.v[2], A2 = s.v[3];
    const double X1 = s.fx[0] + A1 * p2, Y1 = s.fx[1] - A1 * p1;  // Re, Im of D_1 psi
    const double X2 = s.fy[0] + A2 * p2, Y2 = s.fy[1] - A2 * p1;  // Re, Im of D_2 psi
    const double B = s.fx[3] - s.fy[2];
    const double w = u * u - (p1 * p1 + p2 * p2);
    dgx[0] = X1; dgy[0] = X2;
    dgx[1] = Y1; dgy[1] = Y2;
    dgx[3] = B;  dgy[2] = -B;
    dv[0] = -A1 * Y1 - A2 * Y2 - 0.5 * lam * w * p1;
    dv[1] = A1 * X1 + A2 * X2 - 0.5 * lam * w * p2;
    dv[2] = X1 * p2 - Y1 * p1;
    dv[3] = X2 * p2 - Y2 * p1;
  } else if (theory == TH_CHIRAL_MAGNET || theory == TH_CM_DEMAG) {  // demag part added over the lattice
    const double J = prm[0], D = prm[1], K = prm[2], h = prm[3];
    double dv1[3], dv2[3];
    dmi_vectors((int)prm[4], dv1, dv2);
    const double n[3] = {s.v[0], s.v[1], s.v[2]};
    const double nx_[3] = {s.fx[0], s.fx[1], s.fx[2]};
    const double ny_[3] = {s.fy[0], s.fy[1], s.fy[2]};
    // d_i . (n x d_i n) = n . (d_i n x d_i)  = d_i n . (d_i x n)
    double a1[3], a2[3], b1[3], b2[3];
    cross(dv1, n, a1);    // d/d(d_1 n) of the DMI term
    cross(dv2, n, a2);
    cross(nx_, dv1, b1);  // d/dn of the DMI term
    cross(ny_, dv2, b2);
    for (int a = 0; a < 3; ++a) {
      dgx[a] = J * nx_[a] + D * a1[a];
      dgy[a] = J * ny_[a] + D * a2[a];
      dv[a] = D * (b1[a] + b2[a]);
    }
    dv[2] += -2.0 * K * n[2] - h;
  } else if (theory == TH_BABY_SKYRME) {
    const double k2 = prm[0] * prm[0], mu2 = prm[1] * prm[1], nu2 = prm[2] * prm[2];
    const double a[3] = {s.fx[0], s.fx[1], s.fx[2]}, b[3] = {s.fy[0], s.fy[1], s.fy[2]};
    const double aa = dot3(a, a), bb = dot3(b, b), ab = dot3(a, b);
    for (int c = 0; c < 3; ++c) {
      dgx[c] = a[c] + k2 * (bb * a[c] - ab * b[c]);
      dgy[c] = b[c] + k2 * (aa * b[c] - ab * a[c]);
    }
    dv[0] = nu2 * s.v[0];
    dv[2] = -mu2;
  } else if (theory == TH_SID) {
    const double a1 = prm[0], a2 = prm[1], b1 = prm[2], b2 = prm[3], b3 = prm[4], b4 = prm[5], nu = prm[6];
    const SidTerms t = sid_terms(s);
    const double A[2] = {s.v[4], s.v[5]};
    const double eta[2] = {1.0, -1.0};
    double* dg[2] = {dgx, dgy};
    for (int a = 0; a < 2; ++a) {
      const int b = 1 - a;
      const double u = s.v[2 * a], w = s.v[2 * a + 1];
      for (int j = 0; j < 2; ++j) {
        const double P = t.X[a][j] + nu * eta[j] * t.X[b][j], Q = t.Y[a][j] + nu * eta[j] * t.Y[b][j];
        dg[j][2 * a] = P;       // d e / d(d_j u_a)
        dg[j][2 * a + 1] = Q;   // d e / d(d_j w_a)
        dv[2 * a] += -A[j] * Q;
        dv[2 * a + 1] += A[j] * P;
        dv[4 + j] += P * w - Q * u;
      }
    }
    dgx[5] = t.B;
    dgy[4] = -t.B;
    const double s1 = s.v[0], s2 = s.v[1], d1 = s.v[2], d2 = s.v[3];
    dv[0] += 2 * a1 * s1 + 4 * b1 * t.S * s1 + 2 * b3 * t.Dd * s1 + 4 * b4 * (t.p * d1 + t.q * d2);
    dv[1] += 2 * a1 * s2 + 4 * b1 * t.S * s2 + 2 * b3 * t.Dd * s2 + 4 * b4 * (t.p * d2 - t.q * d1);
    dv[2] += 2 * a2 * d1 + 4 * b2 * t.Dd * d1 + 2 * b3 * t.S * d1 + 4 * b4 * (t.p * s1 - t.q * s2);
    dv[3] += 2 * a2 * d2 + 4 * b2 * t.Dd * d2 + 2 * b3 * t.S * d2 + 4 * b4 * (t.p * s2 + t.q * s1);
  } else if (theory == TH_BEC) {
    const double g = prm[0], Om = prm[1], mu = prm[2];
    const double u = s.v[0], v = s.v[1];
    const double Du = s.x * s.fy[0] - s.y * s.fx[0], Dv = s.x * s.fy[1] - s.y * s.fx[1];
    const double w = s.x * s.x + s.y * s.y + 2.0 * g * (u * u + v * v) - 2.0 * mu;
    // -Omega (u D v - v D u): d/d(d_x u) = -Omega v y, d/d(d_y u) = Omega v x,
    // d/d(d_x v) = Omega u y, d/d(d_y v) = -Omega u x, d/du = -Omega D v, d/dv = Omega D u
    dgx[0] = s.fx[0] - Om * v * s.y;  dgy[0] = s.fy[0] + Om * v * s.x;
    dgx[1] = s.fx[1] + Om * u * s.y;  dgy[1] = s.fy[1] - Om * u * s.x;
    dv[0] = w * u - Om * Dv;
    dv[1] = w * v + Om * Du;
  } else {
    dv[0] = prm[0] * s.v[0];
  }
}

// ---------------------------------------------------------------- demagnetisation
// Magnetostatic charge rho = d_1 n_1 + d_2 n_2 (Eq. 1) on I, zero elsewhere.
void demag_charge(const double* f, const Grid& g, double* rho) {
  std::memset(rho, 0, sizeof(double) * g.plane());
  for (int j = 2; j <= g.ny - 3; ++j)
    for (int i = 2; i <= g.nx - 3; ++i) rho[(size_t)j * g.nx + i] = d1x(f, g, i, j) + d1y(f + g.plane(), g, i, j);
}

// The Dirichlet box along one axis of N interior sites: its size N' (the smallest
// N' >= N whose N' + 1 has no prime factor above 7) and the sites it adds below I.
void demag_box(int N, int* Np, int* below) {
  auto smooth = [](int m) {
    for (int q : {2, 3, 5, 7})
      while (m % q == 0) m /= q;
    return m == 1;
  };
  int n = N;
  while (!smooth(n + 1)) ++n;
  *Np = n;
  *below = (n - N) / 2;
}

// Solve L psi = rho on the Dirichlet box (5-point Laplacian, psi = 0 on the nodes
// just outside it) by the sine transform that diagonalises L: box index
// i' = i - 1 + bx = 1..Nx (i' = 0 and Nx + 1 the zero nodes; bx the sites below I),
// L sin(pi k i'/(Nx+1)) sin(pi l j'/(Ny+1)) = lambda_kl (same mode),
//   lambda_kl = -(2 - 2 cos(pi k/(Nx+1)))/dx^2 - (2 - 2 cos(pi l/(Ny+1)))/dy^2,
// with the transform written out as plain sums (test sizes only). box receives psi at
// box nodes [0, Ny + 1] x [0, Nx + 1] (zero on the outer ones); psi (if not null) the
// array plane, psi on I and zero on the halo.
void demag_box_potential(const double* f, const Grid& g, std::vector<double>& box, int& Nx, int& Ny, int& bx,
                         int& by) {
  demag_box(g.nx - 4, &Nx, &bx);
  demag_box(g.ny - 4, &Ny, &by);
  std::vector<double> rho_a(g.plane());
  demag_charge(f, g, rho_a.data());
  // rho on the box: the array's charge on I, zero on the padding
  std::vector<double> rho((size_t)(Nx + 2) * (Ny + 2), 0.0);
  auto bat = [&](int ip, int jp) { return (size_t)jp * (Nx + 2) + ip; };
  for (int j = 2; j <= g.ny - 3; ++j)
    for (int i = 2; i <= g.nx - 3; ++i) rho[bat(i - 1 + bx, j - 1 + by)] = rho_a[(size_t)j * g.nx + i];
  std::vector<double> sx((size_t)Nx * Nx), sy((size_t)Ny * Ny);
  for (int k = 1; k <= Nx; ++k)
    for (int i = 1; i <= Nx; ++i) sx[(size_t)(k - 1) * Nx + (i - 1)] = std::sin(PI * k * i / (Nx + 1));
  for (int l = 1; l <= Ny; ++l)
    for (int j = 1; j <= Ny; ++j) sy[(size_t)(l - 1) * Ny + (j - 1)] = std::sin(PI * l * j / (Ny + 1));
  std::vector<double> a((size_t)Nx * Ny), b((size_t)Nx * Ny);
  for (int jp = 1; jp <= Ny; ++jp)  // along x
    for (int k = 1; k <= Nx; ++k) {
      double acc = 0.0;
      for (int ip = 1; ip <= Nx; ++ip) acc += sx[(size_t)(k - 1) * Nx + (ip - 1)] * rho[bat(ip, jp)];
      a[(size_t)(jp - 1) * Nx + (k - 1)] = acc;
    }
  for (int l = 1; l <= Ny; ++l)  // along y, then divide by the eigenvalue
    for (int k = 1; k <= Nx; ++k) {
      double acc = 0.0;
      for (int jp = 1; jp <= Ny; ++jp) acc += sy[(size_t)(l - 1) * Ny + (jp - 1)] * a[(size_t)(jp - 1) * Nx + (k - 1)];
      const double lam = -(2.0 - 2.0 * std::cos(PI * k / (Nx + 1))) / (g.dx * g.dx) -
                         (2.0 - 2.0 * std::cos(PI * l / (Ny + 1))) / (g.dy * g.dy);
      b[(size_t)(l - 1) * Nx + (k - 1)] = acc / lam;
    }
  const double norm = (2.0 / (Nx + 1)) * (2.0 / (Ny + 1));
  for (int jp = 1; jp <= Ny; ++jp)  // inverse along y
    for (int k = 1; k <= Nx; ++k) {
      double acc = 0.0;
      for (int l = 1; l <= Ny; ++l) acc += sy[(size_t)(l - 1) * Ny + (jp - 1)] * b[(size_t)(l - 1) * Nx + (k - 1)];
      a[(size_t)(jp - 1) * Nx + (k - 1)] = acc;
    }
  box.assign((size_t)(Nx + 2) * (Ny + 2), 0.0);
  for (int jp = 1; jp <= Ny; ++jp)  // inverse along x
    for (int ip = 1; ip <= Nx; ++ip) {
      double acc = 0.0;
      for (int k = 1; k <= Nx; ++k) acc += sx[(size_t)(k - 1) * Nx + (ip - 1)] * a[(size_t)(jp - 1) * Nx + (k - 1)];
      box[bat(ip, jp)] = norm * acc;
    }
}

// psi on I (zero on the halo): the box solution at I's sites.
void demag_potential(const double* f, const Grid& g, double* psi) {
  std::vector<double> box;
  int Nx, Ny, bx, by;
  demag_box_potential(f, g, box, Nx, Ny, bx, by);
  std::memset(psi, 0, sizeof(double) * g.plane());
  for (int j = 2; j <= g.ny - 3; ++j)
    for (int i = 2; i <= g.nx - 3; ++i) psi[(size_t)j * g.nx + i] = box[(size_t)(j - 1 + by) * (Nx + 2) + (i - 1 + bx)];
}

// E_ms = -mu_d/2 dx dy sum_I psi rho.
double demag_energy(const double* prm, const double* f, const Grid& g) {
  std::vector<double> rho(g.plane()), psi(g.plane());
  demag_charge(f, g, rho.data());
  demag_potential(f, g, psi.data());
  Neumaier acc;
  for (int j = 2; j <= g.ny - 3; ++j)
    for (int i = 2; i <= g.nx - 3; ++i) acc.add(psi[(size_t)j * g.nx + i] * rho[(size_t)j * g.nx + i]);
  return -0.5 * prm[5] * g.dx * g.dy * acc.value();
}

// ---------------------------------------------------------------- lattice sums
double energy(int theory, const double* prm, const double* f, const Grid& g) {
  const int C = ncomp(theory);
  std::vector<double> e(g.plane(), 0.0);
#pragma omp parallel for schedule(static)
  for (int j = 2; j <= g.ny - 3; ++j)
    for (int i = 2; i <= g.nx - 3; ++i) e[(size_t)j * g.nx + i] = density(theory, prm, gather(f, C, g, i, j, false));
  Neumaier acc;
  for (int j = 2; j <= g.ny - 3; ++j)
    for (int i = 2; i <= g.nx - 3; ++i) acc.add(e[(size_t)j * g.nx + i]);
  const double E = g.dx * g.dy * acc.value();
  return theory == TH_CM_DEMAG ? E + demag_energy(prm, f, g) : E;
}

// G on I, zero on the halo. Demagnetisation: with the potential psi_in if given (the
// step's held potential), else the potential of f itself.
void force(int theory, const double* prm, const double* f, const Grid& g, double* G, const double* psi_in = nullptr) {
  const int C = ncomp(theory);
  std::memset(G, 0, sizeof(double) * C * g.plane());
  std::vector<double> psi_own;
  const double* psi = psi_in;
  if (theory == TH_CM_DEMAG && !psi) {
    psi_own.resize(g.plane());
    demag_potential(f, g, psi_own.data());
    psi = psi_own.data();
  }
#pragma omp parallel for schedule(static)
  for (int j = 2; j <= g.ny - 3; ++j)
    for (int i = 2; i <= g.nx - 3; ++i) {
      double Gs[6];
      const Site st = gather(f, C, g, i, j, true);
      if (theory == TH_CM_DEMAG) {
        const double pg[2] = {d1x(psi, g, i, j), d1y(psi, g, i, j)};
        force_cm(prm, st, Gs, pg);
      } else {
        force_site(theory, prm, st, Gs);
      }
      for (int c = 0; c < C; ++c) G[c * g.plane() + (size_t)j * g.nx + i] = Gs[c];
    }
}

double max_abs(const double* a, size_t n) {
  double m = 0.0;
  for (size_t k = 0; k < n; ++k) m = std::fmax(m, std::fabs(a[k]));
  return m;
}

// Unit-length projection of the chiral magnet (Sec. 3.2): n <- n / |n| on every
// interior site (the halo is fixed and already unit length).
void normalise(double* f, const Grid& g) {
  const size_t P = g.plane();
  for (int j = 2; j <= g.ny - 3; ++j)
    for (int i = 2; i <= g.nx - 3; ++i) {
      const size_t k = (size_t)j * g.nx + i;
      const double r = std::sqrt(f[k] * f[k] + f[P + k] * f[P + k] + f[2 * P + k] * f[2 * P + k]);
      f[k] /= r; f[P + k] /= r; f[2 * P + k] /= r;
    }
}
// Tangent projection of a velocity: v <- v - (v . n) n.
void tangent(double* v, const double* n, const Grid& g) {
  const size_t P = g.plane();
  for (size_t k = 0; k < P; ++k) {
    const double vn = v[k] * n[k] + v[P + k] * n[P + k] + v[2 * P + k] * n[2 * P + k];
    v[k] -= vn * n[k]; v[P + k] -= vn * n[P + k]; v[2 * P + k] -= vn * n[2 * P + k];
  }
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

int or_ncomp(int theory) { return ncomp(theory); }

// Threads the oracle's parallel loops use (1 without OpenMP).
int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Sec. 3.1: dt = C * dx with the default Courant-like number C = 0.5; with
// unequal spacings the smaller one is used.
double or_time_step(double dx, double dy) { return 0.5 * (dx < dy ? dx : dy); }

// Eq. 1, Eq. 2 and the mixed derivative of one plane on I (zero on the halo).
void or_derivatives(const double* p, int nx, int ny, double dx, double dy, double* fx, double* fy, double* fxx,
                    double* fyy, double* fxy) {
  const Grid g{nx, ny, dx, dy};
  const size_t P = g.plane();
  std::memset(fx, 0, P * 8); std::memset(fy, 0, P * 8); std::memset(fxx, 0, P * 8);
  std::memset(fyy, 0, P * 8); std::memset(fxy, 0, P * 8);
  for (int j = 2; j <= ny - 3; ++j)
    for (int i = 2; i <= nx - 3; ++i) {
      const size_t k = (size_t)j * nx + i;
      fx[k] = d1x(p, g, i, j); fy[k] = d1y(p, g, i, j);
      fxx[k] = d2x(p, g, i, j); fyy[k] = d2y(p, g, i, j); fxy[k] = d12(p, g, i, j);
    }
}

// Energy density e on I (zero on the halo).
void or_energy_density(int theory, const double* prm, const double* f, int nx, int ny, double dx, double dy,
                       double* e) {
  const Grid g{nx, ny, dx, dy};
  const int C = ncomp(theory);
  std::memset(e, 0, sizeof(double) * g.plane());
  for (int j = 2; j <= ny - 3; ++j)
    for (int i = 2; i <= nx - 3; ++i) e[(size_t)j * nx + i] = density(theory, prm, gather(f, C, g, i, j, false));
}

// E_h = dx dy sum_I e  (Sec. 3.2, discretised energy functional).
double or_energy(int theory, const double* prm, const double* f, int nx, int ny, double dx, double dy) {
  return energy(theory, prm, f, Grid{nx, ny, dx, dy});
}

// Euler-Lagrange force G on I (zero on the halo); chiral magnet tangent-projected.
void or_force(int theory, const double* prm, const double* f, int nx, int ny, double dx, double dy, double* G) {
  force(theory, prm, f, Grid{nx, ny, dx, dy}, G);
}

// Demagnetisation: the magnetostatic charge rho and potential psi of a field (both
// [ny][nx], zero off I), and E_ms alone (prm as for the chiral magnet with demag).
void or_demag_potential(const double* f, int nx, int ny, double dx, double dy, double* rho, double* psi) {
  const Grid g{nx, ny, dx, dy};
  demag_charge(f, g, rho);
  demag_potential(f, g, psi);
}
// The Dirichlet box of an axis with N interior sites: out = {N', sites below I}.
void or_demag_box(int N, int* out) { demag_box(N, &out[0], &out[1]); }
// psi on the whole box [Ny' + 2][Nx' + 2] (the zero nodes included); box must hold
// (Nx' + 2)(Ny' + 2) doubles, sizes from or_demag_box.
void or_demag_box_potential(const double* f, int nx, int ny, double dx, double dy, double* box) {
  std::vector<double> b;
  int Nx, Ny, bx, by;
  demag_box_potential(f, Grid{nx, ny, dx, dy}, b, Nx, Ny, bx, by);
  std::memcpy(box, b.data(), sizeof(double) * b.size());
}
double or_demag_energy(const double* prm, const double* f, int nx, int ny, double dx, double dy) {
  return demag_energy(prm, f, Grid{nx, ny, dx, dy});
}

// Exact gradient dE_h/dphi of the lattice energy (adjoint of Eq. 1), no projection.
// Used only to pin G; footprint 9x9 instead of G's 5x5.
void or_energy_grad_exact(int theory, const double* prm, const double* f, int nx, int ny, double dx, double dy,
                          double* grad) {
  const Grid g{nx, ny, dx, dy};
  const int C = ncomp(theory);
  const size_t P = g.plane();
  std::memset(grad, 0, sizeof(double) * C * P);
  const double w[5] = {1.0, -8.0, 0.0, 8.0, -1.0};  // Eq. 1 weights at offsets -2..2
  const double A = dx * dy;
  for (int j = 2; j <= ny - 3; ++j)
    for (int i = 2; i <= nx - 3; ++i) {
      double dv[6], dgx[6], dgy[6];
      partials(theory, prm, gather(f, C, g, i, j, false), dv, dgx, dgy);
      for (int c = 0; c < C; ++c) {
        double* gc = grad + c * P;
        gc[(size_t)j * nx + i] += A * dv[c];
        for (int m = -2; m <= 2; ++m) {
          gc[(size_t)j * nx + (i + m)] += A * dgx[c] * w[m + 2] / (12.0 * dx);
          gc[(size_t)(j + m) * nx + i] += A * dgy[c] * w[m + 2] / (12.0 * dy);
        }
      }
    }
  if (theory == TH_CM_DEMAG) {
    // d E_ms / d n = mu_d dx dy (Eq. 1 gradient of psi) at every site, the halo included
    // (the charges on I see the halo's in-plane values), psi taken as zero off the array
    std::vector<double> psi(g.plane());
    demag_potential(f, g, psi.data());
    auto ps = [&](int i, int j) { return (i < 0 || i >= nx || j < 0 || j >= ny) ? 0.0 : psi[(size_t)j * nx + i]; };
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const double gx = (-ps(i + 2, j) + 8.0 * ps(i + 1, j) - 8.0 * ps(i - 1, j) + ps(i - 2, j)) / (12.0 * dx);
        const double gy = (-ps(i, j + 2) + 8.0 * ps(i, j + 1) - 8.0 * ps(i, j - 1) + ps(i, j - 2)) / (12.0 * dy);
        grad[(size_t)j * nx + i] += A * prm[5] * gx;
        grad[P + (size_t)j * nx + i] += A * prm[5] * gy;
      }
  }
}

}  // extern "C"

namespace {

// The RK4 update of one arrested-Newton-flow step (Eq. 3) by classic RK4 on the
// first-order system (phi, v = phi-dot) (Sec. 3.2), without the arrest:
//   k1 = (v,            -G(phi))
//   k2 = (v + dt/2 k1v, -G(phi + dt/2 k1phi))
//   k3 = (v + dt/2 k2v, -G(phi + dt/2 k2phi))
//   k4 = (v + dt   k3v, -G(phi + dt   k3phi))
//   (phi, v) += dt/6 (k1 + 2 k2 + 2 k3 + k4)
// Chiral magnet: every stage input and phi^{n+1} are normalised; v^{n+1} is
// tangent-projected at phi^{n+1}. Halo sites stay fixed (v = 0 there).
void rk4_update(int theory, const double* prm, double* f, double* v, const Grid& g, double dt) {
  const int C = ncomp(theory);
  const size_t N = (size_t)C * g.plane();
  const bool cm = unit_vector(theory);
  // v and every G vanish on the halo, so every k_phi and k_v does too and the halo
  // stays fixed without special cases.
  std::vector<double> k1p(N), k1v(N), k2p(N), k2v(N), k3p(N), k3v(N), k4p(N), k4v(N), y(N);
  std::vector<double> psi;  // demagnetisation: the potential of phi^n, held through the stages
  if (theory == TH_CM_DEMAG) {
    psi.resize(g.plane());
    demag_potential(f, g, psi.data());
  }
  auto kv_at = [&](std::vector<double>& kv) {  // k_v = -G(y)
    if (cm) normalise(y.data(), g);
    force(theory, prm, y.data(), g, kv.data(), psi.empty() ? nullptr : psi.data());
    for (size_t k = 0; k < N; ++k) kv[k] = -kv[k];
  };
  // k1
  for (size_t k = 0; k < N; ++k) { y[k] = f[k]; k1p[k] = v[k]; }
  kv_at(k1v);
  // k2
  for (size_t k = 0; k < N; ++k) { y[k] = f[k] + 0.5 * dt * k1p[k]; k2p[k] = v[k] + 0.5 * dt * k1v[k]; }
  kv_at(k2v);
  // k3
  for (size_t k = 0; k < N; ++k) { y[k] = f[k] + 0.5 * dt * k2p[k]; k3p[k] = v[k] + 0.5 * dt * k2v[k]; }
  kv_at(k3v);
  // k4
  for (size_t k = 0; k < N; ++k) { y[k] = f[k] + dt * k3p[k]; k4p[k] = v[k] + dt * k3v[k]; }
  kv_at(k4v);
  // combine
  for (size_t k = 0; k < N; ++k) {
    f[k] += dt / 6.0 * (k1p[k] + 2.0 * k2p[k] + 2.0 * k3p[k] + k4p[k]);
    v[k] += dt / 6.0 * (k1v[k] + 2.0 * k2v[k] + 2.0 * k3v[k] + k4v[k]);
  }
  if (cm) {
    normalise(f, g);
    tangent(v, f, g);
  }
}

}  // namespace

extern "C" {

// One arrested-Newton-flow step (Eq. 3, Eq. 4): the RK4 update above, then, if
// E_h(phi^{n+1}) > E_h(phi^n), v^{n+1} <- 0 (Eq. 4).
// *E_io holds E_h(phi^n) on entry and E_h(phi^{n+1}) on exit. Returns 1 if arrested.
int or_anf_step(int theory, const double* prm, double* f, double* v, int nx, int ny, double dx, double dy, double dt,
                double* E_io) {
  const Grid g{nx, ny, dx, dy};
  const int C = ncomp(theory);
  const size_t N = (size_t)C * g.plane();
  rk4_update(theory, prm, f, v, g, dt);
  const double E_new = energy(theory, prm, f, g);
  int arrested = 0;
  if (E_new > *E_io) {  // Eq. 4, strict
    std::memset(v, 0, sizeof(double) * N);
    arrested = 1;
  }
  *E_io = E_new;
  return arrested;
}

// Arrested Newton flow from the given (phi, v) until max_I |dx dy G(phi)| < tol or
// max_steps steps have been taken. out = {E, norm (dx dy max|G|), steps, arrests}.
// Returns 1 if converged, 0 otherwise.
int or_minimise(int theory, const double* prm, double* f, double* v, int nx, int ny, double dx, double dy, double dt,
                double tol, long long max_steps, double* out) {
  const Grid g{nx, ny, dx, dy};
  const int C = ncomp(theory);
  const size_t N = (size_t)C * g.plane();
  std::vector<double> G(N);
  double E = energy(theory, prm, f, g);
  long long steps = 0, arrests = 0;
  double norm = 0.0;
  int converged = 0;
  for (;;) {
    force(theory, prm, f, g, G.data());
    norm = dx * dy * max_abs(G.data(), N);
    if (norm < tol) { converged = 1; break; }
    if (steps >= max_steps) break;
    arrests += or_anf_step(theory, prm, f, v, nx, ny, dx, dy, dt, &E);
    ++steps;
  }
  out[0] = E; out[1] = norm; out[2] = (double)steps; out[3] = (double)arrests;
  return converged;
}

// ---------------------------------------------------------------- gradient descent
// The first-order alternative of Sec. 3.2: descent along -grad E_h without
// fictitious inertia. The paper names it but gives no scheme; it is read here as
// the explicit Euler step of the gradient flow  d phi / d tau = -G(phi):
//   phi^{n+1} = phi^n - dtau G(phi^n)   on I (the halo stays fixed),
// the chiral magnet renormalised to |n| = 1 afterwards (the projection the arrested
// flow applies to its new field). Nothing is arrested; an energy increase
// E_h(phi^{n+1}) > E_h(phi^n) is only counted (it means dtau is past the stability
// limit). *E_io holds E_h(phi^n) on entry and E_h(phi^{n+1}) on exit; returns 1 if
// the energy rose.
int or_gd_step(int theory, const double* prm, double* f, int nx, int ny, double dx, double dy, double dtau,
               double* E_io) {
  const Grid g{nx, ny, dx, dy};
  const int C = ncomp(theory);
  const size_t N = (size_t)C * g.plane();
  std::vector<double> G(N);
  force(theory, prm, f, g, G.data());  // zero on the halo (demagnetisation: psi of phi^n)
  for (size_t k = 0; k < N; ++k) f[k] -= dtau * G[k];
  if (unit_vector(theory)) normalise(f, g);
  const double E_new = energy(theory, prm, f, g);
  const int rose = E_new > *E_io ? 1 : 0;
  *E_io = E_new;
  return rose;
}

// Stability limit of that Euler step for the stencil Laplacian: Eq. 2 has the
// symbol -(30 - 32 cos t + 2 cos 2t) / (12 h^2) along each axis, largest in
// magnitude at t = pi (16 / (3 h^2)), so -lap has the largest eigenvalue
// lambda = (16/3)(1/dx^2 + 1/dy^2) and the step is stable for dtau < 2 / lambda.
double or_gd_step_limit(double dx, double dy) { return 2.0 / ((16.0 / 3.0) * (1.0 / (dx * dx) + 1.0 / (dy * dy))); }

// Gradient descent from phi until max_I |dx dy G(phi)| < tol or max_steps steps.
// out = {E, norm (dx dy max|G|), steps, energy rises}. Returns 1 if converged.
int or_gd_minimise(int theory, const double* prm, double* f, int nx, int ny, double dx, double dy, double dtau,
                   double tol, long long max_steps, double* out) {
  const Grid g{nx, ny, dx, dy};
  const int C = ncomp(theory);
  const size_t N = (size_t)C * g.plane();
  std::vector<double> G(N);
  double E = energy(theory, prm, f, g);
  long long steps = 0, rises = 0;
  double norm = 0.0;
  int converged = 0;
  for (;;) {
    force(theory, prm, f, g, G.data());
    norm = dx * dy * max_abs(G.data(), N);
    if (norm < tol) { converged = 1; break; }
    if (steps >= max_steps) break;
    rises += or_gd_step(theory, prm, f, nx, ny, dx, dy, dtau, &E);
    ++steps;
  }
  out[0] = E; out[1] = norm; out[2] = (double)steps; out[3] = (double)rises;
  return converged;
}

// ---------------------------------------------------------------- BEC at a fixed atom number
// The BEC section holds the atom number N = int |psi|^2 fixed (its normalisation).
// Read here as the flow on the constraint surface N_h(psi) = dx dy sum_I |psi|^2 = N0
// of the lattice functional at zero chemical potential, E_h = dx dy sum_I e(mu = 0):
//   refresh of a new field (psi, v):
//     v   <- v - alpha psi on I,  alpha = sum_I v.psi / sum_I |psi|^2  (v tangent to the
//            constraint surface; psi and the scaled psi point the same way),
//     psi <- s psi on I,  s = sqrt(N0 / N_h(psi))  (the halo keeps its values),
//     mu  =  sum_I G_0(psi).psi / (2 sum_I |psi|^2)  for the scaled psi, G_0 the force at
//            zero chemical potential: the Lagrange multiplier of the constraint, for which
//            the force G_mu = G_0 - 2 mu psi of the grand-canonical form has no part along
//            psi (the part the constraint removes);
//   one step: the BEC flow at chemical potential mu (held through the RK stages, like
//     the potential of the demagnetising field), then a refresh;
//   arrest (Eq. 4) and convergence as for every theory, on E_h at mu = 0 and on
//     dx dy max_I |G_mu| of the refreshed field.
// Gradient descent takes the same refresh after each Euler step (v absent).
namespace {

double bec_sum_sq(const double* f, const Grid& g) {  // sum_I |psi|^2
  const size_t P = g.plane();
  Neumaier a;
  for (int j = 2; j <= g.ny - 3; ++j)
    for (int i = 2; i <= g.nx - 3; ++i) {
      const size_t k = (size_t)j * g.nx + i;
      a.add(f[k] * f[k] + f[P + k] * f[P + k]);
    }
  return a.value();
}

// mu = sum_I G_0.psi / (2 sum_I |psi|^2); prm = {g, Omega, ...} (its mu is not used)
double bec_multiplier(const double* prm, const double* f, const Grid& g) {
  const double p0[3] = {prm[0], prm[1], 0.0};
  const size_t P = g.plane();
  std::vector<double> G(2 * P);
  force(TH_BEC, p0, f, g, G.data());
  Neumaier a;
  for (size_t k = 0; k < P; ++k) a.add(G[k] * f[k] + G[P + k] * f[P + k]);  // G = 0 off I
  return a.value() / (2.0 * bec_sum_sq(f, g));
}

// The refresh above; v may be null (gradient descent). Returns 0, or -1 if N_h(psi)
// is zero or not finite (nothing to scale).
int bec_refresh(const double* prm, double N0, double* f, double* v, const Grid& g, double* mu) {
  const size_t P = g.plane();
  const double S = bec_sum_sq(f, g);
  if (!(S > 0.0) || !std::isfinite(S)) return -1;
  if (v) {
    Neumaier vp;
    for (int j = 2; j <= g.ny - 3; ++j)
      for (int i = 2; i <= g.nx - 3; ++i) {
        const size_t k = (size_t)j * g.nx + i;
        vp.add(v[k] * f[k] + v[P + k] * f[P + k]);
      }
    const double alpha = vp.value() / S;
    for (int j = 2; j <= g.ny - 3; ++j)
      for (int i = 2; i <= g.nx - 3; ++i) {
        const size_t k = (size_t)j * g.nx + i;
        v[k] -= alpha * f[k];
        v[P + k] -= alpha * f[P + k];
      }
  }
  const double sc = std::sqrt(N0 / (g.dx * g.dy * S));
  for (int j = 2; j <= g.ny - 3; ++j)
    for (int i = 2; i <= g.nx - 3; ++i) {
      const size_t k = (size_t)j * g.nx + i;
      f[k] *= sc;
      f[P + k] *= sc;
    }
  *mu = bec_multiplier(prm, f, g);
  return 0;
}

}  // namespace

// The multiplier of a field as it stands (no scaling).
double or_bec_multiplier(const double* prm, const double* f, int nx, int ny, double dx, double dy) {
  return bec_multiplier(prm, f, Grid{nx, ny, dx, dy});
}

// The refresh of a new field; v may be NULL. Returns 0 or -1 (see bec_refresh).
int or_bec_refresh(const double* prm, double N0, double* f, double* v, int nx, int ny, double dx, double dy,
                   double* mu) {
  return bec_refresh(prm, N0, f, v, Grid{nx, ny, dx, dy}, mu);
}

// One step at fixed atom number from a refreshed (psi, v) whose multiplier is *mu_io
// and energy (mu = 0) *E_io: the RK4 update at chemical potential mu, the refresh,
// then Eq. 4 on E_h at mu = 0. On exit *mu_io and *E_io belong to the new field.
// Returns 1 if arrested, 0 if not, -1 if the refresh failed.
int or_anf_step_fixed_n(const double* prm, double N0, double* f, double* v, int nx, int ny, double dx, double dy,
                        double dt, double* E_io, double* mu_io) {
  const Grid g{nx, ny, dx, dy};
  const double pm[3] = {prm[0], prm[1], *mu_io}, p0[3] = {prm[0], prm[1], 0.0};
  rk4_update(TH_BEC, pm, f, v, g, dt);
  if (bec_refresh(prm, N0, f, v, g, mu_io) != 0) return -1;
  const double E_new = energy(TH_BEC, p0, f, g);
  int arrested = 0;
  if (E_new > *E_io) {
    std::memset(v, 0, sizeof(double) * 2 * g.plane());
    arrested = 1;
  }
  *E_io = E_new;
  return arrested;
}

// Arrested Newton flow at fixed atom number N0 from (phi, v), refreshed first, until
// dx dy max_I |G_mu| < tol or max_steps steps. out = {E (mu = 0), norm, steps,
// arrests, mu}. Returns 1 if converged, 0 if not, -1 if a refresh failed.
int or_minimise_fixed_n(const double* prm, double N0, double* f, double* v, int nx, int ny, double dx, double dy,
                        double dt, double tol, long long max_steps, double* out) {
  const Grid g{nx, ny, dx, dy};
  const size_t N = 2 * g.plane();
  std::vector<double> G(N);
  double mu = 0.0;
  if (bec_refresh(prm, N0, f, v, g, &mu) != 0) return -1;
  const double p0[3] = {prm[0], prm[1], 0.0};
  double E = energy(TH_BEC, p0, f, g);
  long long steps = 0, arrests = 0;
  double norm = 0.0;
  int converged = 0;
  for (;;) {
    const double pm[3] = {prm[0], prm[1], mu};
    force(TH_BEC, pm, f, g, G.data());
    norm = dx * dy * max_abs(G.data(), N);
    if (norm < tol) { converged = 1; break; }
    if (steps >= max_steps) break;
    const int a = or_anf_step_fixed_n(prm, N0, f, v, nx, ny, dx, dy, dt, &E, &mu);
    if (a < 0) return -1;
    arrests += a;
    ++steps;
  }
  out[0] = E; out[1] = norm; out[2] = (double)steps; out[3] = (double)arrests; out[4] = mu;
  return converged;
}

// Gradient descent at fixed atom number: phi <- phi - dtau G_mu(phi), then the refresh
// (no velocity); rises of E_h (mu = 0) are counted. out as for or_minimise_fixed_n
// with out[3] = energy rises.
int or_gd_minimise_fixed_n(const double* prm, double N0, double* f, int nx, int ny, double dx, double dy,
                           double dtau, double tol, long long max_steps, double* out) {
  const Grid g{nx, ny, dx, dy};
  const size_t N = 2 * g.plane();
  std::vector<double> G(N);
  double mu = 0.0;
  if (bec_refresh(prm, N0, f, nullptr, g, &mu) != 0) return -1;
  const double p0[3] = {prm[0], prm[1], 0.0};
  double E = energy(TH_BEC, p0, f, g);
  long long steps = 0, rises = 0;
  double norm = 0.0;
  int converged = 0;
  for (;;) {
    const double pm[3] = {prm[0], prm[1], mu};
    force(TH_BEC, pm, f, g, G.data());
    norm = dx * dy * max_abs(G.data(), N);
    if (norm < tol) { converged = 1; break; }
    if (steps >= max_steps) break;
    for (size_t k = 0; k < N; ++k) f[k] -= dtau * G[k];
    if (bec_refresh(prm, N0, f, nullptr, g, &mu) != 0) return -1;
    const double E_new = energy(TH_BEC, p0, f, g);
    rises += E_new > E ? 1 : 0;
    E = E_new;
    ++steps;
  }
  out[0] = E; out[1] = norm; out[2] = (double)steps; out[3] = (double)rises; out[4] = mu;
  return converged;
}

// Signed solid angle of the spherical triangle (a, b, c):
// tan(Omega/2) = a.(b x c) / (1 + a.b + b.c + c.a)   (Berg and Luescher, 1981).
static double solid_angle(const double a[3], const double b[3], const double c[3]) {
  double bc[3];
  cross(b, c, bc);
  return 2.0 * std::atan2(dot3(a, bc), 1.0 + dot3(a, b) + dot3(b, c) + dot3(c, a));
}

// Observables (Sec. 2 "GPU-resident evaluation of observables"; Sec. 3.3):
// out[0] = E_h
// out[1] = topological charge: chiral magnet Berg-Luescher lattice charge over all
//          plaquettes, two triangles each, oriented like n.(d_1 n x d_2 n), divided by
//          4 pi; Abelian Higgs winding of arg psi around the boundary of I
//          (counter-clockwise), divided by 2 pi.
// out[2] = magnetic flux dx dy sum_I (d_1 A_2 - d_2 A_1) (Abelian Higgs, s+id), 0 otherwise
// out[3] = dx dy max_I |G|, out[4] = max_I |G|
// out[5] = max over all sites of ||n| - 1| (chiral magnet, Baby Skyrme), 0 otherwise
// out[6] = BEC atom number N = dx dy sum_I |psi|^2, out[7] = BEC angular momentum
//          dx dy sum_I Re(psi* L_z psi); 0 otherwise
void or_observables(int theory, const double* prm, const double* f, int nx, int ny, double dx, double dy,
                    double* out) {
  const Grid g{nx, ny, dx, dy};
  const int C = ncomp(theory);
  const size_t P = g.plane(), N = (size_t)C * P;
  std::vector<double> G(N);
  force(theory, prm, f, g, G.data());
  const double gmax = max_abs(G.data(), N);
  out[0] = energy(theory, prm, f, g);
  out[1] = 0.0; out[2] = 0.0; out[3] = dx * dy * gmax; out[4] = gmax; out[5] = 0.0; out[6] = 0.0; out[7] = 0.0;
  if (theory == TH_BEC) {
    Neumaier na, lz;
    for (int j = 2; j <= ny - 3; ++j)
      for (int i = 2; i <= nx - 3; ++i) {
        const Site s = gather(f, 2, g, i, j, false);
        na.add(s.v[0] * s.v[0] + s.v[1] * s.v[1]);
        lz.add(s.v[0] * (s.x * s.fy[1] - s.y * s.fx[1]) - s.v[1] * (s.x * s.fy[0] - s.y * s.fx[0]));
      }
    out[6] = dx * dy * na.value();
    out[7] = dx * dy * lz.value();
  }
  if (unit_vector(theory)) {
    auto unit = [&](int i, int j, double n[3]) {
      const size_t k = (size_t)j * nx + i;
      const double r = std::sqrt(f[k] * f[k] + f[P + k] * f[P + k] + f[2 * P + k] * f[2 * P + k]);
      n[0] = f[k] / r; n[1] = f[P + k] / r; n[2] = f[2 * P + k] / r;
    };
    Neumaier q;
    for (int j = 0; j + 1 < ny; ++j)
      for (int i = 0; i + 1 < nx; ++i) {
        double n00[3], n10[3], n11[3], n01[3];
        unit(i, j, n00); unit(i + 1, j, n10); unit(i + 1, j + 1, n11); unit(i, j + 1, n01);
        q.add(solid_angle(n00, n10, n11));
        q.add(solid_angle(n00, n11, n01));
      }
    out[1] = q.value() / (4.0 * PI);
    double dev = 0.0;
    for (size_t k = 0; k < P; ++k)
      dev = std::fmax(dev, std::fabs(std::sqrt(f[k] * f[k] + f[P + k] * f[P + k] + f[2 * P + k] * f[2 * P + k]) - 1.0));
    out[5] = dev;
  } else if (theory == TH_ABELIAN_HIGGS || theory == TH_SID) {
    // loop of boundary sites of I, counter-clockwise (s+id: the winding of Delta_s)
    std::vector<int> li, lj;
    for (int i = 2; i < nx - 3; ++i) { li.push_back(i); lj.push_back(2); }
    for (int j = 2; j < ny - 3; ++j) { li.push_back(nx - 3); lj.push_back(j); }
    for (int i = nx - 3; i > 2; --i) { li.push_back(i); lj.push_back(ny - 3); }
    for (int j = ny - 3; j > 2; --j) { li.push_back(2); lj.push_back(j); }
    Neumaier w;
    const size_t L = li.size();
    for (size_t k = 0; k < L; ++k) {
      const size_t a = (size_t)lj[k] * nx + li[k], b = (size_t)lj[(k + 1) % L] * nx + li[(k + 1) % L];
      double d = std::atan2(f[P + b], f[b]) - std::atan2(f[P + a], f[a]);
      while (d > PI) d -= 2.0 * PI;
      while (d <= -PI) d += 2.0 * PI;
      w.add(d);
    }
    out[1] = w.value() / (2.0 * PI);
    Neumaier flux;
    const double* A1 = f + (theory == TH_SID ? 4 : 2) * P;
    const double* A2 = f + (theory == TH_SID ? 5 : 3) * P;
    for (int j = 2; j <= ny - 3; ++j)
      for (int i = 2; i <= nx - 3; ++i) flux.add(d1x(A2, g, i, j) - d1y(A1, g, i, j));
    out[2] = dx * dy * flux.value();
  }
}

// Initial configurations ("model-specific ansatz", Sec. 3.4 / Sec. 4.1). The paper
// gives no formula; these are the standard forms.
// Abelian Higgs, product of unit-size radial vortices of winding n_k at (x_k, y_k):
//   psi = prod_k tanh(r_k/s_k)^{|n_k|} exp(i (n_k theta_k + chi_k)),
//   A   = sum_k n_k tanh^2(r_k/s_k) (-(y-y_k), x-x_k) / r_k^2   (A = 0 at r_k = 0).
// Chiral magnet, compact skyrmions of radius R_k = s_k, vorticity m_k, helicity gamma_k:
//   n = (sin f cos(m theta + gamma), sin f sin(m theta + gamma), cos f),
//   f = pi (1 - r/R) for r < R, else 0 (n = e_3); the first disc containing a site wins.
// sol[k*5 + 0..4] = {x, y, charge, size, phase}.
// BEC: Thomas-Fermi amplitude times vortex factors,
//   psi = sqrt(max(0, mu - r^2/2) / g) prod_k tanh(r_k/s_k)^{|n_k|} exp(i (n_k theta_k + chi_k)).
void or_ansatz_bec(const double* prm, const double* sol, int nsol, double* f, int nx, int ny, double dx, double dy) {
  const size_t P = (size_t)nx * ny;
  const double g = prm[0], mu = prm[2];
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double x = (i - 0.5 * (nx - 1)) * dx, y = (j - 0.5 * (ny - 1)) * dy;
      double mod = std::sqrt(std::fmax(0.0, mu - 0.5 * (x * x + y * y)) / g), ph = 0.0;
      for (int s = 0; s < nsol; ++s) {
        const double X = x - sol[5 * s], Y = y - sol[5 * s + 1];
        const double n = sol[5 * s + 2], sz = sol[5 * s + 3], chi = sol[5 * s + 4];
        mod *= std::pow(std::tanh(std::sqrt(X * X + Y * Y) / sz), std::fabs(n));
        ph += n * std::atan2(Y, X) + chi;
      }
      const size_t k = (size_t)j * nx + i;
      f[k] = mod * std::cos(ph);
      f[P + k] = mod * std::sin(ph);
    }
}

// s+id: the uniform minimum of the potential over S = |Delta_s|^2, D = |Delta_d|^2 >= 0 with
// the relative phase phi that minimises b4 (Ds^2 conj(Dd)^2 + c.c.) = 2 b4 S D cos(2 phi)
// (phi = pi/2 for b4 > 0, else 0), then Delta_s = sqrt(S) w, Delta_d = sqrt(D) e^{i phi} w,
// with w = prod_k tanh(r_k/s_k)^{|n_k|} e^{i (n_k theta_k + chi_k)}, and A as for the
// Abelian Higgs vortices. out_min (may be NULL) receives {S, D, phi}.
void or_ansatz_sid(const double* prm, const double* sol, int nsol, double* f, int nx, int ny, double dx, double dy,
                   double* out_min) {
  const double a1 = prm[0], a2 = prm[1], b1 = prm[2], b2 = prm[3], b4 = prm[5];
  const double phi = b4 > 0.0 ? 0.5 * PI : 0.0;
  const double c = prm[4] + 2.0 * b4 * std::cos(2.0 * phi);  // effective S D coefficient
  auto V = [&](double S, double D) { return a1 * S + a2 * D + b1 * S * S + b2 * D * D + c * S * D; };
  double S = 0.0, D = 0.0, best = 0.0;
  // candidates: the interior stationary point and the two one-band minima
  const double det = 4.0 * b1 * b2 - c * c;
  double cand[3][2] = {{det != 0.0 ? (c * a2 - 2.0 * b2 * a1) / det : -1.0, det != 0.0 ? (c * a1 - 2.0 * b1 * a2) / det : -1.0},
                       {-a1 / (2.0 * b1), 0.0},
                       {0.0, -a2 / (2.0 * b2)}};
  for (auto& q : cand)
    if (q[0] >= 0.0 && q[1] >= 0.0 && V(q[0], q[1]) < best) { S = q[0]; D = q[1]; best = V(S, D); }
  if (out_min) { out_min[0] = S; out_min[1] = D; out_min[2] = phi; }
  const size_t P = (size_t)nx * ny;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double x = (i - 0.5 * (nx - 1)) * dx, y = (j - 0.5 * (ny - 1)) * dy;
      double mod = 1.0, ph = 0.0, A1 = 0.0, A2 = 0.0;
      for (int k = 0; k < nsol; ++k) {
        const double X = x - sol[5 * k], Y = y - sol[5 * k + 1];
        const double n = sol[5 * k + 2], sz = sol[5 * k + 3], chi = sol[5 * k + 4];
        const double r2 = X * X + Y * Y;
        const double t = std::tanh(std::sqrt(r2) / sz);
        mod *= std::pow(t, std::fabs(n));
        ph += n * std::atan2(Y, X) + chi;
        if (r2 > 0.0) {
          A1 += n * t * t * (-Y) / r2;
          A2 += n * t * t * X / r2;
        }
      }
      const size_t q = (size_t)j * nx + i;
      f[q] = std::sqrt(S) * mod * std::cos(ph);
      f[P + q] = std::sqrt(S) * mod * std::sin(ph);
      f[2 * P + q] = std::sqrt(D) * mod * std::cos(ph + phi);
      f[3 * P + q] = std::sqrt(D) * mod * std::sin(ph + phi);
      f[4 * P + q] = A1;
      f[5 * P + q] = A2;
    }
}

void or_ansatz(int theory, const double* sol, int nsol, double* f, int nx, int ny, double dx, double dy) {
  const size_t P = (size_t)nx * ny;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double x = (i - 0.5 * (nx - 1)) * dx, y = (j - 0.5 * (ny - 1)) * dy;
      const size_t k = (size_t)j * nx + i;
      if (theory == TH_ABELIAN_HIGGS) {
        double mod = 1.0, ph = 0.0, A1 = 0.0, A2 = 0.0;
        for (int s = 0; s < nsol; ++s) {
          const double X = x - sol[5 * s], Y = y - sol[5 * s + 1];
          const double n = sol[5 * s + 2], sz = sol[5 * s + 3], chi = sol[5 * s + 4];
          const double r2 = X * X + Y * Y, r = std::sqrt(r2);
          const double t = std::tanh(r / sz);
          mod *= std::pow(t, std::fabs(n));
          ph += n * std::atan2(Y, X) + chi;
          if (r2 > 0.0) {
            A1 += n * t * t * (-Y) / r2;
            A2 += n * t * t * X / r2;
          }
        }
        f[k] = mod * std::cos(ph);
        f[P + k] = mod * std::sin(ph);
        f[2 * P + k] = A1;
        f[3 * P + k] = A2;
      } else if (unit_vector(theory)) {
        double n1 = 0.0, n2 = 0.0, n3 = 1.0;
        for (int s = 0; s < nsol; ++s) {
          const double X = x - sol[5 * s], Y = y - sol[5 * s + 1];
          const double m = sol[5 * s + 2], R = sol[5 * s + 3], gam = sol[5 * s + 4];
          const double r = std::sqrt(X * X + Y * Y);
          if (r < R) {
            const double fr = PI * (1.0 - r / R), th = m * std::atan2(Y, X) + gam;
            n1 = std::sin(fr) * std::cos(th);
            n2 = std::sin(fr) * std::sin(th);
            n3 = std::cos(fr);
            break;
          }
        }
        f[k] = n1; f[P + k] = n2; f[2 * P + k] = n3;
      }
    }
}

}  // extern "C"
