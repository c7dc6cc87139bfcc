// FP64 CPU oracle for the differentiable structural FEM hot path.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark may load this library.  It shares no code,
// header, table or helper with the CUDA path.  It is written to be read against
// the paper, not to be fast: one element at a time, plain loops, full 24 x 24
// matrix products, and a band Cholesky solve.
//
// What it computes (arXiv 2407.20026, JAX-SSO):
//  * Element stiffness matrices k_e(x) of the beam-column and of the MITC-4
//    quad shell (Sec. 2.2.1).  The paper names them but does not print them;
//    the formulations here are the textbook ones, with these conventions:
//      - DOF order per node (ux, uy, uz, rx, ry, rz), the order of the support
//        and load vectors of Listing 1.
//      - Beam: 3D Euler-Bernoulli frame element, Iy for bending in the local
//        x-z plane and Iz in the local x-y plane; local x along i -> j,
//        local y = unit(e_Z x local x), or e_Y when the member is within
//        1e-8 of vertical; local z = x cross y.
//      - Quad: flat facet on the mean plane of the 4 nodes (normal from the
//        cross product of the diagonals, origin at the centroid, local x along
//        the projection of (X1 - X0) + (X2 - X3)), bilinear plane-stress
//        membrane, Reissner-Mindlin bending, Dvorkin-Bathe assumed transverse
//        shear tied at the 4 edge mid-points (MITC-4), a drilling penalty
//        gamma_d * int (rz - (v_x - u_y)/2)^2 dA with gamma_d = 0.01 G t, all
//        integrated with 2 x 2 Gauss points; shear factor 5/6.  Warped
//        elements: nodes are tied to their projections on the mean plane by
//        rigid links (offset h_i along the normal).
//      - kappa_x, kappa_y scale the membrane and bending rigidities along the
//        local axes (xx by kappa_x, yy by kappa_y, the coupling and in-plane
//        shear terms by sqrt(kappa_x kappa_y)).
//  * Consistent nodal loads of an area load q = pressure + gamma * t acting in
//    -Z: f_i = -q int N_i dA on the flat facet (2 x 2 Gauss).
//  * Global K u = f (Eq. 1) with supports imposed either by deleting the fixed
//    rows and columns (homogeneous supports, b = 0) or by the Lagrange
//    multiplier system K_aug u_aug = f_aug with V u = b (Eqs. 2-3).
//  * Material volume W = sum_e A_e t_e of the quads (Sec. 3.3) with dW/dz and
//    dW/dt, A_e the facet area above.
//  * Compliance C = f^T u and the adjoint sensitivity (Eqs. 5-6):
//    K^T lambda = dJ/du and dJ/dp = dJ/dp|explicit - lambda^T (dK/dp u - df/dp),
//    for J = w C + g^T u.  dk_e/dp comes from forward-mode dual numbers
//    evaluated through the same element routine (Sec. 2.1.1, AD of k_e(x)).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Forward-mode dual number: value and one tangent.
struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double tan_(double) { return 0.0; }
inline double tan_(const Dual& x) { return x.d; }
using std::sqrt;

template <class S>
void cross3(const S a[3], const S b[3], S c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
template <class S>
S dot3(const S a[3], const S b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// K <- T^T K T for an n x n matrix and a block-diagonal T made of (n/3)
// copies of the 3 x 3 rotation R (rows = local axes in global coordinates).
template <class S, int N>
void rotate_to_global(const S R[3][3], S K[N][N]) {
  S T[N][N], tmp[N][N];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) T[i][j] = S(0.0);
  for (int b = 0; b < N / 3; ++b)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) T[3 * b + i][3 * b + j] = R[i][j];
  // tmp = K T
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      S s(0.0);
      for (int k = 0; k < N; ++k) s += K[i][k] * T[k][j];
      tmp[i][j] = s;
    }
  // K = T^T tmp
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      S s(0.0);
      for (int k = 0; k < N; ++k) s += T[k][i] * tmp[k][j];
      K[i][j] = s;
    }
}

// ---------------------------------------------------------------------------
// Beam-column (Sec. 2.2.1, Listing 1: add_beamcol(E, G, Iy, Iz, J, A)).
// p = {E, G, Iy, Iz, J, A}.  K is the 12 x 12 global stiffness.
template <class S>
void beam_ke(const S xi[3], const S xj[3], const S p[6], S K[12][12]) {
  const S E = p[0], G = p[1], Iy = p[2], Iz = p[3], J = p[4], A = p[5];
  S d[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
  S L = sqrt(dot3(d, d));
  S ex[3] = {d[0] / L, d[1] / L, d[2] / L};
  S ey[3], ez[3];
  if (std::fabs(val(ex[2])) > 1.0 - 1e-8) {
    ey[0] = S(0.0); ey[1] = S(1.0); ey[2] = S(0.0);
  } else {
    // e_Z x ex = (-ex_y, ex_x, 0)
    S hx = -ex[1], hy = ex[0];
    S hn = sqrt(hx * hx + hy * hy);
    ey[0] = hx / hn; ey[1] = hy / hn; ey[2] = S(0.0);
  }
  cross3(ex, ey, ez);

  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) K[i][j] = S(0.0);
  S L2 = L * L, L3 = L2 * L;
  S ka = E * A / L, kt = G * J / L;
  K[0][0] = ka; K[6][6] = ka; K[0][6] = -ka;
  K[3][3] = kt; K[9][9] = kt; K[3][9] = -kt;
  // bending in local x-y (v, rz) with Iz
  {
    S a = S(12.0) * E * Iz / L3, b = S(6.0) * E * Iz / L2;
    S c = S(4.0) * E * Iz / L, e = S(2.0) * E * Iz / L;
    K[1][1] = a;  K[1][5] = b;   K[1][7] = -a; K[1][11] = b;
    K[5][5] = c;  K[5][7] = -b;  K[5][11] = e;
    K[7][7] = a;  K[7][11] = -b;
    K[11][11] = c;
  }
  // bending in local x-z (w, ry) with Iy
  {
    S a = S(12.0) * E * Iy / L3, b = S(6.0) * E * Iy / L2;
    S c = S(4.0) * E * Iy / L, e = S(2.0) * E * Iy / L;
    K[2][2] = a;  K[2][4] = -b;  K[2][8] = -a; K[2][10] = -b;
    K[4][4] = c;  K[4][8] = b;   K[4][10] = e;
    K[8][8] = a;  K[8][10] = b;
    K[10][10] = c;
  }
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < i; ++j) K[i][j] = K[j][i];
  S R[3][3];
  for (int k = 0; k < 3; ++k) { R[0][k] = ex[k]; R[1][k] = ey[k]; R[2][k] = ez[k]; }
  rotate_to_global<S, 12>(R, K);
}

// ---------------------------------------------------------------------------
// MITC-4 quad shell (Sec. 2.2.1: a_quad = (x, y, z, t, E, nu, kx, ky)).
const double XI_N[4] = {-1.0, 1.0, 1.0, -1.0};
const double ETA_N[4] = {-1.0, -1.0, 1.0, 1.0};
const double GAUSS = 0.57735026918962576451;  // 1 / sqrt(3)

// Local geometry of the flat facet.
template <class S>
void quad_frame(const S X[4][3], S R[3][3], S xl[4], S yl[4], S hl[4]) {
  S c[3];
  for (int k = 0; k < 3; ++k) c[k] = (X[0][k] + X[1][k] + X[2][k] + X[3][k]) * S(0.25);
  S d13[3], d24[3], nv[3];
  for (int k = 0; k < 3; ++k) { d13[k] = X[2][k] - X[0][k]; d24[k] = X[3][k] - X[1][k]; }
  cross3(d13, d24, nv);
  S nn = sqrt(dot3(nv, nv));
  S n[3] = {nv[0] / nn, nv[1] / nn, nv[2] / nn};
  S a[3];
  for (int k = 0; k < 3; ++k) a[k] = (X[1][k] - X[0][k]) + (X[2][k] - X[3][k]);
  S an = dot3(a, n);
  for (int k = 0; k < 3; ++k) a[k] = a[k] - an * n[k];
  S al = sqrt(dot3(a, a));
  S e1[3] = {a[0] / al, a[1] / al, a[2] / al};
  S e2[3];
  cross3(n, e1, e2);
  for (int k = 0; k < 3; ++k) { R[0][k] = e1[k]; R[1][k] = e2[k]; R[2][k] = n[k]; }
  for (int i = 0; i < 4; ++i) {
    S r[3] = {X[i][0] - c[0], X[i][1] - c[1], X[i][2] - c[2]};
    xl[i] = dot3(r, e1);
    yl[i] = dot3(r, e2);
    hl[i] = dot3(r, n);
  }
}

// Shape functions and the Jacobian of the flat facet at (xi, eta).
template <class S>
struct Pt {
  double N[4], Nxi[4], Neta[4];
  S xxi, yxi, xeta, yeta, detJ;
  S Nx[4], Ny[4];
};

template <class S>
Pt<S> eval_point(const S xl[4], const S yl[4], double xi, double eta) {
  Pt<S> P;
  for (int i = 0; i < 4; ++i) {
    P.N[i] = 0.25 * (1.0 + XI_N[i] * xi) * (1.0 + ETA_N[i] * eta);
    P.Nxi[i] = 0.25 * XI_N[i] * (1.0 + ETA_N[i] * eta);
    P.Neta[i] = 0.25 * ETA_N[i] * (1.0 + XI_N[i] * xi);
  }
  P.xxi = S(0.0); P.yxi = S(0.0); P.xeta = S(0.0); P.yeta = S(0.0);
  for (int i = 0; i < 4; ++i) {
    P.xxi += S(P.Nxi[i]) * xl[i];
    P.yxi += S(P.Nxi[i]) * yl[i];
    P.xeta += S(P.Neta[i]) * xl[i];
    P.yeta += S(P.Neta[i]) * yl[i];
  }
  P.detJ = P.xxi * P.yeta - P.yxi * P.xeta;
  // [N_x; N_y] = J^{-1} [N_xi; N_eta],  J = [[x_xi, y_xi], [x_eta, y_eta]]
  for (int i = 0; i < 4; ++i) {
    P.Nx[i] = (P.yeta * S(P.Nxi[i]) - P.yxi * S(P.Neta[i])) / P.detJ;
    P.Ny[i] = (-P.xeta * S(P.Nxi[i]) + P.xxi * S(P.Neta[i])) / P.detJ;
  }
  return P;
}

// K += w * B^T D B for B (m x 24) and D (m x m).
template <class S, int M>
void add_btdb(S K[24][24], const S B[M][24], const S D[M][M], S w) {
  for (int i = 0; i < 24; ++i)
    for (int j = 0; j < 24; ++j) {
      S s(0.0);
      for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b) s += B[a][i] * D[a][b] * B[b][j];
      K[i][j] += w * s;
    }
}

// Covariant transverse shear rows at a tying point (MITC-4, Dvorkin-Bathe):
// g_xi = w_xi + beta . x_xi and g_eta = w_eta + beta . x_eta with
// beta_x = ry, beta_y = -rx.
template <class S>
void covariant_shear(const S xl[4], const S yl[4], double xi, double eta,
                     S gxi[24], S geta[24]) {
  Pt<S> P = eval_point(xl, yl, xi, eta);
  for (int j = 0; j < 24; ++j) { gxi[j] = S(0.0); geta[j] = S(0.0); }
  for (int i = 0; i < 4; ++i) {
    gxi[6 * i + 2] = S(P.Nxi[i]);
    gxi[6 * i + 3] = -S(P.N[i]) * P.yxi;
    gxi[6 * i + 4] = S(P.N[i]) * P.xxi;
    geta[6 * i + 2] = S(P.Neta[i]);
    geta[6 * i + 3] = -S(P.N[i]) * P.yeta;
    geta[6 * i + 4] = S(P.N[i]) * P.xeta;
  }
}

// p = {t, E, nu, kappa_x, kappa_y}.  K is the 24 x 24 global stiffness.
template <class S>
void quad_ke(const S X[4][3], const S p[5], S K[24][24]) {
  const S t = p[0], E = p[1], nu = p[2], kx = p[3], ky = p[4];
  S R[3][3], xl[4], yl[4], hl[4];
  quad_frame(X, R, xl, yl, hl);

  const S G = E / (S(2.0) * (S(1.0) + nu));
  const S kxy = sqrt(kx * ky);
  const S cm = E * t / (S(1.0) - nu * nu);
  const S cb = E * t * t * t / (S(12.0) * (S(1.0) - nu * nu));
  S Dm[3][3], Db[3][3], Ds[2][2], Dd[1][1];
  const S pat[3][3] = {{kx, nu * kxy, S(0.0)},
                       {nu * kxy, ky, S(0.0)},
                       {S(0.0), S(0.0), kxy * (S(1.0) - nu) * S(0.5)}};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) { Dm[a][b] = cm * pat[a][b]; Db[a][b] = cb * pat[a][b]; }
  Ds[0][0] = S(5.0 / 6.0) * G * t; Ds[0][1] = S(0.0);
  Ds[1][0] = S(0.0);               Ds[1][1] = S(5.0 / 6.0) * G * t;
  Dd[0][0] = S(0.01) * G * t;

  // tying points: B=(0,-1), D=(0,+1) for g_xi;  A=(-1,0), C=(+1,0) for g_eta
  S gxiB[24], getaB[24], gxiD[24], getaD[24], gxiA[24], getaA[24], gxiC[24], getaC[24];
  covariant_shear(xl, yl, 0.0, -1.0, gxiB, getaB);
  covariant_shear(xl, yl, 0.0, 1.0, gxiD, getaD);
  covariant_shear(xl, yl, -1.0, 0.0, gxiA, getaA);
  covariant_shear(xl, yl, 1.0, 0.0, gxiC, getaC);

  S Kf[24][24];
  for (int i = 0; i < 24; ++i)
    for (int j = 0; j < 24; ++j) Kf[i][j] = S(0.0);

  for (int gj = 0; gj < 2; ++gj)
    for (int gi = 0; gi < 2; ++gi) {
      const double xi = (gi == 0 ? -GAUSS : GAUSS);
      const double eta = (gj == 0 ? -GAUSS : GAUSS);
      Pt<S> P = eval_point(xl, yl, xi, eta);
      S Bm[3][24], Bb[3][24], Bs[2][24], Bd[1][24];
      for (int a = 0; a < 3; ++a)
        for (int j = 0; j < 24; ++j) { Bm[a][j] = S(0.0); Bb[a][j] = S(0.0); }
      for (int j = 0; j < 24; ++j) { Bs[0][j] = S(0.0); Bs[1][j] = S(0.0); Bd[0][j] = S(0.0); }
      for (int i = 0; i < 4; ++i) {
        // membrane: eps = [u_x, v_y, u_y + v_x]
        Bm[0][6 * i + 0] = P.Nx[i];
        Bm[1][6 * i + 1] = P.Ny[i];
        Bm[2][6 * i + 0] = P.Ny[i];
        Bm[2][6 * i + 1] = P.Nx[i];
        // bending: kappa = [bx_x, by_y, bx_y + by_x], bx = ry, by = -rx
        Bb[0][6 * i + 4] = P.Nx[i];
        Bb[1][6 * i + 3] = -P.Ny[i];
        Bb[2][6 * i + 3] = -P.Nx[i];
        Bb[2][6 * i + 4] = P.Ny[i];
        // drilling: rz - (v_x - u_y) / 2
        Bd[0][6 * i + 0] = S(0.5) * P.Ny[i];
        Bd[0][6 * i + 1] = S(-0.5) * P.Nx[i];
        Bd[0][6 * i + 5] = S(P.N[i]);
      }
      // assumed covariant shear, then to Cartesian with J^{-1}
      for (int j = 0; j < 24; ++j) {
        S gxi = S(0.5 * (1.0 - eta)) * gxiB[j] + S(0.5 * (1.0 + eta)) * gxiD[j];
        S geta = S(0.5 * (1.0 - xi)) * getaA[j] + S(0.5 * (1.0 + xi)) * getaC[j];
        Bs[0][j] = (P.yeta * gxi - P.yxi * geta) / P.detJ;
        Bs[1][j] = (-P.xeta * gxi + P.xxi * geta) / P.detJ;
      }
      add_btdb<S, 3>(Kf, Bm, Dm, P.detJ);
      add_btdb<S, 3>(Kf, Bb, Db, P.detJ);
      add_btdb<S, 2>(Kf, Bs, Ds, P.detJ);
      add_btdb<S, 1>(Kf, Bd, Dd, P.detJ);
    }

  // rigid links to the mean plane: u_P = u - h ry, v_P = v + h rx
  S W[24][24], tmp[24][24];
  for (int i = 0; i < 24; ++i)
    for (int j = 0; j < 24; ++j) W[i][j] = S(i == j ? 1.0 : 0.0);
  for (int i = 0; i < 4; ++i) {
    W[6 * i + 0][6 * i + 4] = -hl[i];
    W[6 * i + 1][6 * i + 3] = hl[i];
  }
  for (int i = 0; i < 24; ++i)
    for (int j = 0; j < 24; ++j) {
      S s(0.0);
      for (int k = 0; k < 24; ++k) s += Kf[i][k] * W[k][j];
      tmp[i][j] = s;
    }
  for (int i = 0; i < 24; ++i)
    for (int j = 0; j < 24; ++j) {
      S s(0.0);
      for (int k = 0; k < 24; ++k) s += W[k][i] * tmp[k][j];
      K[i][j] = s;
    }
  rotate_to_global<S, 24>(R, K);
}

// Consistent nodal load of the area load q (N/m^2) acting in -Z.
template <class S>
void quad_fe(const S X[4][3], S q, S f[24]) {
  S R[3][3], xl[4], yl[4], hl[4];
  quad_frame(X, R, xl, yl, hl);
  for (int j = 0; j < 24; ++j) f[j] = S(0.0);
  for (int gj = 0; gj < 2; ++gj)
    for (int gi = 0; gi < 2; ++gi) {
      const double xi = (gi == 0 ? -GAUSS : GAUSS);
      const double eta = (gj == 0 ? -GAUSS : GAUSS);
      Pt<S> P = eval_point(xl, yl, xi, eta);
      for (int i = 0; i < 4; ++i) f[6 * i + 2] -= q * S(P.N[i]) * P.detJ;
    }
}

template <class S>
S quad_area(const S X[4][3]) {
  S R[3][3], xl[4], yl[4], hl[4];
  quad_frame(X, R, xl, yl, hl);
  S a(0.0);
  for (int gj = 0; gj < 2; ++gj)
    for (int gi = 0; gi < 2; ++gi) {
      Pt<S> P = eval_point(xl, yl, gi == 0 ? -GAUSS : GAUSS, gj == 0 ? -GAUSS : GAUSS);
      a += P.detJ;
    }
  return a;
}

}  // namespace

// ===========================================================================
// C interface (ctypes).
extern "C" {

typedef struct {
  int32_t n_nodes;
  const double* xyz;          // [n_nodes * 3]
  int32_t n_beams;
  const int32_t* beam_conn;   // [n_beams * 2]
  const double* beam_props;   // [n_beams * 6]  E, G, Iy, Iz, J, A
  int32_t n_quads;
  const int32_t* quad_conn;   // [n_quads * 4]
  const double* quad_props;   // [n_quads * 5]  t, E, nu, kx, ky
  const uint8_t* fixed;       // [n_nodes * 6]
  const double* nodal_load;   // [n_nodes * 6]
  double pressure;            // Pa, -Z
  double gamma;               // N/m^3 self weight, -Z
} orc_mesh;

enum { ORC_OK = 0, ORC_ERR_INVALID = 1, ORC_ERR_SINGULAR = 3, ORC_ERR_NOT_CONVERGED = 4 };

void orc_beam_ke(const double* xi, const double* xj, const double* props, double* ke) {
  double K[12][12];
  beam_ke<double>(xi, xj, props, K);
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) ke[12 * i + j] = K[i][j];
}

// d k_e / d p for one scalar input p: which = 0..2 -> xi[which], 6..8 ->
// xj[which-6], 12..17 -> props[which-12] (3..5 and 9..11 are unused).
void orc_beam_dke(const double* xi, const double* xj, const double* props, int which,
                  double* dke) {
  Dual a[3], b[3], p[6], K[12][12];
  for (int k = 0; k < 3; ++k) { a[k] = Dual(xi[k], which == k); b[k] = Dual(xj[k], which == 6 + k); }
  for (int k = 0; k < 6; ++k) p[k] = Dual(props[k], which == 12 + k);
  beam_ke<Dual>(a, b, p, K);
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) dke[12 * i + j] = K[i][j].d;
}

void orc_quad_ke(const double* X, const double* props, double* ke) {
  double Xn[4][3], K[24][24];
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 3; ++k) Xn[i][k] = X[3 * i + k];
  quad_ke<double>(Xn, props, K);
  for (int i = 0; i < 24; ++i)
    for (int j = 0; j < 24; ++j) ke[24 * i + j] = K[i][j];
}

// which = 0..11 -> X[which] (node which/3, axis which%3); 12..16 -> props.
void orc_quad_dke(const double* X, const double* props, int which, double* dke) {
  Dual Xn[4][3], p[5], K[24][24];
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 3; ++k) Xn[i][k] = Dual(X[3 * i + k], which == 3 * i + k);
  for (int k = 0; k < 5; ++k) p[k] = Dual(props[k], which == 12 + k);
  quad_ke<Dual>(Xn, p, K);
  for (int i = 0; i < 24; ++i)
    for (int j = 0; j < 24; ++j) dke[24 * i + j] = K[i][j].d;
}

void orc_quad_fe(const double* X, double q, double* fe) {
  double Xn[4][3], f[24];
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 3; ++k) Xn[i][k] = X[3 * i + k];
  quad_fe<double>(Xn, q, f);
  for (int j = 0; j < 24; ++j) fe[j] = f[j];
}

double orc_quad_area(const double* X) {
  double Xn[4][3];
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 3; ++k) Xn[i][k] = X[3 * i + k];
  return quad_area<double>(Xn);
}

}  // extern "C"

namespace {

void quad_nodes(const orc_mesh* m, int e, double X[4][3]) {
  for (int a = 0; a < 4; ++a) {
    int n = m->quad_conn[4 * e + a];
    for (int k = 0; k < 3; ++k) X[a][k] = m->xyz[3 * n + k];
  }
}

// Full (unconstrained) load vector: nodal loads plus consistent area loads.
std::vector<double> full_load(const orc_mesh* m) {
  const int n = 6 * m->n_nodes;
  std::vector<double> f(m->nodal_load, m->nodal_load + n);
  for (int e = 0; e < m->n_quads; ++e) {
    double X[4][3], fe[24];
    quad_nodes(m, e, X);
    const double q = m->pressure + m->gamma * m->quad_props[5 * e + 0];
    quad_fe<double>(X, q, fe);
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 6; ++d) f[6 * m->quad_conn[4 * e + a] + d] += fe[6 * a + d];
  }
  return f;
}

// Calls fn(global dofs[], n, ke[n*n]) for every element.
template <class F>
void for_each_element(const orc_mesh* m, F fn) {
  for (int e = 0; e < m->n_beams; ++e) {
    int ni = m->beam_conn[2 * e], nj = m->beam_conn[2 * e + 1];
    double K[12][12];
    beam_ke<double>(m->xyz + 3 * ni, m->xyz + 3 * nj, m->beam_props + 6 * e, K);
    int dofs[12];
    for (int d = 0; d < 6; ++d) { dofs[d] = 6 * ni + d; dofs[6 + d] = 6 * nj + d; }
    fn(dofs, 12, &K[0][0]);
  }
  for (int e = 0; e < m->n_quads; ++e) {
    double X[4][3], K[24][24];
    quad_nodes(m, e, X);
    quad_ke<double>(X, m->quad_props + 5 * e, K);
    int dofs[24];
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 6; ++d) dofs[6 * a + d] = 6 * m->quad_conn[4 * e + a] + d;
    fn(dofs, 24, &K[0][0]);
  }
}

// Symmetric positive definite band matrix (lower band, row-major:
// B[i*(bw+1) + (j - i + bw)] = K[i][j] for i - bw <= j <= i) and its Cholesky
// factor stored in place.
struct Band {
  int n = 0, bw = 0;
  std::vector<double> a;
  double& at(int i, int j) { return a[(size_t)i * (bw + 1) + (j - i + bw)]; }
  double get(int i, int j) const { return a[(size_t)i * (bw + 1) + (j - i + bw)]; }
  int factor() {
    for (int i = 0; i < n; ++i) {
      const int lo = std::max(0, i - bw);
      for (int j = lo; j <= i; ++j) {
        const int klo = std::max(lo, j - bw);
        double s = at(i, j);
        const double* ri = &a[(size_t)i * (bw + 1) + (klo - i + bw)];
        const double* rj = &a[(size_t)j * (bw + 1) + (klo - j + bw)];
        for (int k = 0; k < j - klo; ++k) s -= ri[k] * rj[k];
        if (i == j) {
          if (!(s > 0.0)) return ORC_ERR_SINGULAR;
          at(i, i) = std::sqrt(s);
        } else {
          at(i, j) = s / at(j, j);
        }
      }
    }
    return ORC_OK;
  }
  void solve(std::vector<double>& x) const {
    for (int i = 0; i < n; ++i) {  // L y = b
      double s = x[i];
      for (int j = std::max(0, i - bw); j < i; ++j) s -= get(i, j) * x[j];
      x[i] = s / get(i, i);
    }
    for (int i = n - 1; i >= 0; --i) {  // L^T x = y
      double s = x[i];
      for (int j = i + 1; j <= std::min(n - 1, i + bw); ++j) s -= get(j, i) * x[j];
      x[i] = s / get(i, i);
    }
  }
};

// Reduced system K_ff over the free DOFs (fixed rows and columns deleted).
struct Reduced {
  std::vector<int> free_of;   // full dof -> free index or -1
  std::vector<int> full_of;   // free index -> full dof
  Band band;
};

int build_reduced(const orc_mesh* m, Reduced& R) {
  const int n = 6 * m->n_nodes;
  R.free_of.assign(n, -1);
  R.full_of.clear();
  for (int i = 0; i < n; ++i)
    if (!m->fixed[i]) { R.free_of[i] = (int)R.full_of.size(); R.full_of.push_back(i); }
  const int nf = (int)R.full_of.size();
  int bw = 0;
  for_each_element(m, [&](const int* dofs, int nd, const double*) {
    int lo = 1 << 30, hi = -1;
    for (int a = 0; a < nd; ++a) {
      int f = R.free_of[dofs[a]];
      if (f >= 0) { lo = std::min(lo, f); hi = std::max(hi, f); }
    }
    if (hi >= 0) bw = std::max(bw, hi - lo);
  });
  R.band.n = nf;
  R.band.bw = bw;
  R.band.a.assign((size_t)nf * (bw + 1), 0.0);
  for_each_element(m, [&](const int* dofs, int nd, const double* ke) {
    for (int a = 0; a < nd; ++a) {
      int fa = R.free_of[dofs[a]];
      if (fa < 0) continue;
      for (int b = 0; b < nd; ++b) {
        int fb = R.free_of[dofs[b]];
        if (fb < 0 || fb > fa) continue;
        R.band.at(fa, fb) += ke[a * nd + b];
      }
    }
  });
  return R.band.factor();
}

// Dense LU with partial pivoting; solves A x = b in place (A is n x n).
int dense_lu_solve(int n, std::vector<double>& A, std::vector<double>& b) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * n + k]) > best) { best = std::fabs(A[(size_t)i * n + k]); p = i; }
    if (best == 0.0) return ORC_ERR_SINGULAR;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      A[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
      b[i] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[(size_t)i * n + j] * b[j];
    b[i] = s / A[(size_t)i * n + i];
  }
  return ORC_OK;
}

// Sum over elements of -lambda_e^T (dk_e/dp) u_e + mu_e^T (df_e/dp), mu =
// lambda + w u, for p = the z coordinate of every node and the thickness of
// every quad (Eq. 6 with dJ/dp|explicit = w u^T df/dp folded into mu).
void adjoint_contract(const orc_mesh* m, const std::vector<double>& u,
                      const std::vector<double>& lam, double w, double* dz, double* dt) {
  for (int i = 0; i < m->n_nodes; ++i) dz[i] = 0.0;
  for (int e = 0; e < m->n_quads; ++e) dt[e] = 0.0;
  for (int e = 0; e < m->n_beams; ++e) {
    const int nodes[2] = {m->beam_conn[2 * e], m->beam_conn[2 * e + 1]};
    for (int which = 0; which < 2; ++which) {
      Dual a[3], b[3], p[6], K[12][12];
      for (int k = 0; k < 3; ++k) {
        a[k] = Dual(m->xyz[3 * nodes[0] + k], (which == 0 && k == 2) ? 1.0 : 0.0);
        b[k] = Dual(m->xyz[3 * nodes[1] + k], (which == 1 && k == 2) ? 1.0 : 0.0);
      }
      for (int k = 0; k < 6; ++k) p[k] = Dual(m->beam_props[6 * e + k]);
      beam_ke<Dual>(a, b, p, K);
      double s = 0.0;
      for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j)
          s += lam[6 * nodes[i / 6] + i % 6] * K[i][j].d * u[6 * nodes[j / 6] + j % 6];
      dz[nodes[which]] -= s;
    }
  }
  for (int e = 0; e < m->n_quads; ++e) {
    int nodes[4];
    for (int a = 0; a < 4; ++a) nodes[a] = m->quad_conn[4 * e + a];
    for (int which = 0; which < 5; ++which) {
      Dual X[4][3], p[5], K[24][24], f[24];
      for (int a = 0; a < 4; ++a)
        for (int k = 0; k < 3; ++k)
          X[a][k] = Dual(m->xyz[3 * nodes[a] + k], (which == a && k == 2) ? 1.0 : 0.0);
      for (int k = 0; k < 5; ++k) p[k] = Dual(m->quad_props[5 * e + k], (which == 4 && k == 0) ? 1.0 : 0.0);
      quad_ke<Dual>(X, p, K);
      Dual q = Dual(m->pressure) + Dual(m->gamma) * p[0];
      quad_fe<Dual>(X, q, f);
      double s = 0.0;
      for (int i = 0; i < 24; ++i) {
        const int gi = 6 * nodes[i / 6] + i % 6;
        double ki = 0.0;
        for (int j = 0; j < 24; ++j) ki += K[i][j].d * u[6 * nodes[j / 6] + j % 6];
        s += -lam[gi] * ki + (lam[gi] + w * u[gi]) * f[i].d;
      }
      if (which < 4) dz[nodes[which]] += s; else dt[e] += s;
    }
  }
}

}  // namespace

extern "C" {

// Full load vector (nodal + consistent area loads), length 6 n_nodes.
void orc_load_vector(const orc_mesh* m, double* f) {
  std::vector<double> v = full_load(m);
  std::copy(v.begin(), v.end(), f);
}

// Dense global stiffness, no supports, (6 n_nodes)^2 entries.  Small meshes.
void orc_assemble_dense(const orc_mesh* m, double* K) {
  const int n = 6 * m->n_nodes;
  std::fill(K, K + (size_t)n * n, 0.0);
  for_each_element(m, [&](const int* dofs, int nd, const double* ke) {
    for (int a = 0; a < nd; ++a)
      for (int b = 0; b < nd; ++b) K[(size_t)dofs[a] * n + dofs[b]] += ke[a * nd + b];
  });
}

// r = f - K u on every DOF, with r = 0 on fixed DOFs.  Element by element.
void orc_residual(const orc_mesh* m, const double* u, double* r) {
  std::vector<double> f = full_load(m);
  const int n = 6 * m->n_nodes;
  for (int i = 0; i < n; ++i) r[i] = f[i];
  for_each_element(m, [&](const int* dofs, int nd, const double* ke) {
    for (int a = 0; a < nd; ++a) {
      double s = 0.0;
      for (int b = 0; b < nd; ++b) s += ke[a * nd + b] * u[dofs[b]];
      r[dofs[a]] -= s;
    }
  });
  for (int i = 0; i < n; ++i)
    if (m->fixed[i]) r[i] = 0.0;
}

// Half bandwidth of K_ff in the natural (node-major) free-DOF numbering.
int orc_half_bandwidth(const orc_mesh* m) {
  Reduced R;
  const int n = 6 * m->n_nodes;
  R.free_of.assign(n, -1);
  int nf = 0;
  for (int i = 0; i < n; ++i)
    if (!m->fixed[i]) R.free_of[i] = nf++;
  int bw = 0;
  for_each_element(m, [&](const int* dofs, int nd, const double*) {
    int lo = 1 << 30, hi = -1;
    for (int a = 0; a < nd; ++a) {
      int f = R.free_of[dofs[a]];
      if (f >= 0) { lo = std::min(lo, f); hi = std::max(hi, f); }
    }
    if (hi >= 0) bw = std::max(bw, hi - lo);
  });
  return bw;
}

// Solve K u = f under the supports (Eqs. 1-3, b = 0).
//   method 0: delete fixed rows/columns, band Cholesky of K_ff
//   method 1: delete fixed rows/columns, dense LU with partial pivoting
//   method 2: Lagrange multipliers, K_aug = [[K, V^T], [V, 0]], dense LU
// u has 6 n_nodes entries (zero on fixed DOFs); *C = f^T u.
int orc_solve(const orc_mesh* m, int method, double* u, double* C) {
  const int n = 6 * m->n_nodes;
  std::vector<double> f = full_load(m);
  std::fill(u, u + n, 0.0);
  if (method == 0) {
    Reduced R;
    int st = build_reduced(m, R);
    if (st) return st;
    std::vector<double> x(R.full_of.size());
    for (size_t k = 0; k < x.size(); ++k) x[k] = f[R.full_of[k]];
    R.band.solve(x);
    for (size_t k = 0; k < x.size(); ++k) u[R.full_of[k]] = x[k];
  } else if (method == 1) {
    std::vector<int> full_of;
    for (int i = 0; i < n; ++i)
      if (!m->fixed[i]) full_of.push_back(i);
    const int nf = (int)full_of.size();
    std::vector<double> Kfull((size_t)n * n);
    orc_assemble_dense(m, Kfull.data());
    std::vector<double> A((size_t)nf * nf), b(nf);
    for (int a = 0; a < nf; ++a) {
      b[a] = f[full_of[a]];
      for (int c = 0; c < nf; ++c) A[(size_t)a * nf + c] = Kfull[(size_t)full_of[a] * n + full_of[c]];
    }
    int st = dense_lu_solve(nf, A, b);
    if (st) return st;
    for (int a = 0; a < nf; ++a) u[full_of[a]] = b[a];
  } else if (method == 2) {
    std::vector<int> fixed_dofs;
    for (int i = 0; i < n; ++i)
      if (m->fixed[i]) fixed_dofs.push_back(i);
    const int nc = (int)fixed_dofs.size(), na = n + nc;
    std::vector<double> Kfull((size_t)n * n);
    orc_assemble_dense(m, Kfull.data());
    std::vector<double> A((size_t)na * na, 0.0), b(na, 0.0);
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) A[(size_t)a * na + c] = Kfull[(size_t)a * n + c];
    for (int k = 0; k < nc; ++k) {  // V has a single 1 per constrained DOF
      A[(size_t)(n + k) * na + fixed_dofs[k]] = 1.0;
      A[(size_t)fixed_dofs[k] * na + (n + k)] = 1.0;
    }
    for (int a = 0; a < n; ++a) b[a] = f[a];  // f_aug = (f, b = 0)
    int st = dense_lu_solve(na, A, b);
    if (st) return st;
    for (int a = 0; a < n; ++a) u[a] = b[a];
  } else {
    return ORC_ERR_INVALID;
  }
  double c = 0.0;
  for (int i = 0; i < n; ++i) c += f[i] * u[i];
  *C = c;
  return ORC_OK;
}

// Solve, then the adjoint sensitivity of J = w C + g^T u (Eqs. 5-6):
// K lambda = w f + g (lambda = w u when g is NULL), and
// dJ/dz (per node), dJ/dt (per quad).  u, lam may be NULL.
int orc_gradient(const orc_mesh* m, double w, const double* g, double* u_out, double* C_out,
                 double* dz, double* dt, double* lam_out) {
  const int n = 6 * m->n_nodes;
  std::vector<double> f = full_load(m);
  Reduced R;
  int st = build_reduced(m, R);
  if (st) return st;
  const size_t nf = R.full_of.size();
  std::vector<double> x(nf), u(n, 0.0), lam(n, 0.0);
  for (size_t k = 0; k < nf; ++k) x[k] = f[R.full_of[k]];
  R.band.solve(x);
  for (size_t k = 0; k < nf; ++k) u[R.full_of[k]] = x[k];
  double C = 0.0;
  for (int i = 0; i < n; ++i) C += f[i] * u[i];
  for (int i = 0; i < n; ++i) lam[i] = w * u[i];
  if (g) {
    std::vector<double> y(nf);
    for (size_t k = 0; k < nf; ++k) y[k] = g[R.full_of[k]];
    R.band.solve(y);
    for (size_t k = 0; k < nf; ++k) lam[R.full_of[k]] += y[k];
  }
  adjoint_contract(m, u, lam, w, dz, dt);
  if (u_out) std::copy(u.begin(), u.end(), u_out);
  if (C_out) *C_out = C;
  if (lam_out) std::copy(lam.begin(), lam.end(), lam_out);
  return ORC_OK;
}

// The adjoint contraction alone for given u and lambda (no solve).
void orc_adjoint_contract(const orc_mesh* m, const double* u, const double* lam, double w,
                          double* dz, double* dt) {
  const int n = 6 * m->n_nodes;
  std::vector<double> uu(u, u + n), ll(lam, lam + n);
  adjoint_contract(m, uu, ll, w, dz, dt);
}

// dJ/dE_j per quad for J = w C + g^T u at a given (u, lambda): the stiffness
// term -lambda_e^T (dk_e/dE) u_e of Eq. 6 (loads do not depend on E), dk_e/dE by
// dual numbers seeded on the element's Young's modulus.  With SIMP (Eq.
// simp_eq, E_j = p_j^P E*_j) the caller forms dJ/dp_j = dJ/dE_j P p_j^(P-1) E*_j.
void orc_adjoint_contract_E(const orc_mesh* m, const double* u, const double* lam, double* dE) {
  for (int e = 0; e < m->n_quads; ++e) {
    int nodes[4];
    for (int a = 0; a < 4; ++a) nodes[a] = m->quad_conn[4 * e + a];
    Dual X[4][3], p[5], K[24][24];
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 3; ++k) X[a][k] = Dual(m->xyz[3 * nodes[a] + k]);
    for (int k = 0; k < 5; ++k) p[k] = Dual(m->quad_props[5 * e + k], k == 1 ? 1.0 : 0.0);
    quad_ke<Dual>(X, p, K);
    double s = 0.0;
    for (int i = 0; i < 24; ++i)
      for (int j = 0; j < 24; ++j)
        s += lam[6 * nodes[i / 6] + i % 6] * K[i][j].d * u[6 * nodes[j / 6] + j % 6];
    dE[e] = -s;
  }
}

// Material volume of the quads, W = sum_e A_e t_e (Sec. 3.3, the volume term
// of the size-optimisation objective without its minimum-thickness penalty),
// with A_e the area of the element's flat facet (the same 2 x 2 Gauss
// integral as the area loads).  dW/dz per node by dual numbers seeded on that
// node's z in every quad that contains it; dW/dt_e = A_e.
void orc_volume(const orc_mesh* m, double* V, double* dz, double* dt) {
  double vol = 0.0;
  for (int i = 0; i < m->n_nodes; ++i) dz[i] = 0.0;
  for (int e = 0; e < m->n_quads; ++e) {
    int nodes[4];
    for (int a = 0; a < 4; ++a) nodes[a] = m->quad_conn[4 * e + a];
    const double t = m->quad_props[5 * e + 0];
    for (int which = 0; which < 4; ++which) {
      Dual X[4][3];
      for (int a = 0; a < 4; ++a)
        for (int k = 0; k < 3; ++k)
          X[a][k] = Dual(m->xyz[3 * nodes[a] + k], (which == a && k == 2) ? 1.0 : 0.0);
      const Dual A = quad_area<Dual>(X);
      dz[nodes[which]] += t * A.d;
      if (which == 0) {
        dt[e] = A.v;
        vol += A.v * t;
      }
    }
  }
  *V = vol;
}

// Jacobi-preconditioned FP64 CG on K_ff (element-by-element products with
// element matrices computed once), for meshes too large for the band solver.
// Stops when ||f - K u|| <= rtol ||f|| over the free DOFs.  Serial.
int orc_cg(const orc_mesh* m, double rtol, int max_iter, double* u, int* iters) {
  const int n = 6 * m->n_nodes;
  std::vector<double> f = full_load(m);
  for (int i = 0; i < n; ++i)
    if (m->fixed[i]) f[i] = 0.0;
  // element matrices and dof lists
  std::vector<std::vector<int>> edofs;
  std::vector<std::vector<double>> eks;
  for_each_element(m, [&](const int* dofs, int nd, const double* ke) {
    edofs.emplace_back(dofs, dofs + nd);
    eks.emplace_back(ke, ke + nd * nd);
  });
  std::vector<double> diag(n, 0.0);
  for (size_t e = 0; e < edofs.size(); ++e) {
    const int nd = (int)edofs[e].size();
    for (int a = 0; a < nd; ++a) diag[edofs[e][a]] += eks[e][a * nd + a];
  }
  auto matvec = [&](const std::vector<double>& x, std::vector<double>& y) {
    std::fill(y.begin(), y.end(), 0.0);
    for (size_t e = 0; e < edofs.size(); ++e) {
      const int nd = (int)edofs[e].size();
      const int* d = edofs[e].data();
      const double* k = eks[e].data();
      for (int a = 0; a < nd; ++a) {
        if (m->fixed[d[a]]) continue;
        double s = 0.0;
        for (int b = 0; b < nd; ++b)
          if (!m->fixed[d[b]]) s += k[a * nd + b] * x[d[b]];
        y[d[a]] += s;
      }
    }
  };
  std::vector<double> x(n, 0.0), r(f), z(n), p(n), q(n);
  double fn = 0.0;
  for (int i = 0; i < n; ++i) fn += f[i] * f[i];
  fn = std::sqrt(fn);
  for (int i = 0; i < n; ++i) z[i] = m->fixed[i] ? 0.0 : r[i] / diag[i];
  p = z;
  double rz = 0.0;
  for (int i = 0; i < n; ++i) rz += r[i] * z[i];
  int it = 0, st = ORC_ERR_NOT_CONVERGED;
  for (; it < max_iter; ++it) {
    double rr = 0.0;
    for (int i = 0; i < n; ++i) rr += r[i] * r[i];
    if (std::sqrt(rr) <= rtol * fn) { st = ORC_OK; break; }
    matvec(p, q);
    double pq = 0.0;
    for (int i = 0; i < n; ++i) pq += p[i] * q[i];
    if (!(pq > 0.0)) { st = ORC_ERR_SINGULAR; break; }
    const double alpha = rz / pq;
    for (int i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
    for (int i = 0; i < n; ++i) z[i] = m->fixed[i] ? 0.0 : r[i] / diag[i];
    double rz2 = 0.0;
    for (int i = 0; i < n; ++i) rz2 += r[i] * z[i];
    const double beta = rz2 / rz;
    rz = rz2;
    for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
  std::copy(x.begin(), x.end(), u);
  *iters = it;
  return st;
}

}  // extern "C"
