// Element kernels: beam-column and MITC-4 quad stiffness (FP64), consistent
// area loads, and the per-element adjoint contractions of Eq. 6.
//
// Element definitions (arXiv 2407.20026 Sec. 2.2.1 names them; the
// formulations are the textbook ones with these conventions):
//  * DOF order per node (ux, uy, uz, rx, ry, rz) (Listing 1).
//  * Beam: 3D Euler-Bernoulli frame; props (E, G, Iy, Iz, J, A); Iy bends in
//    the local x-z plane, Iz in x-y; local x = (xj - xi)/L, local y =
//    unit(e_Z x local x) or e_Y for a member within 1e-8 of vertical.
//  * Quad: flat facet on the mean plane (normal = unit(d13 x d24) of the
//    diagonals, origin at the centroid, local x along the projection of
//    (X1 - X0) + (X2 - X3)); plane-stress membrane, Reissner-Mindlin bending
//    (beta_x = ry, beta_y = -rx), Dvorkin-Bathe covariant shear tied at the
//    edge mid-points, drilling penalty 0.01 G t (rz - (v_x - u_y)/2)^2, all
//    with 2x2 Gauss points; shear factor 5/6; kappa_x, kappa_y scale the
//    membrane/bending rigidities.  Warped nodes are linked rigidly to their
//    projections: u_P = u - h ry, v_P = v + h rx (local axes).
//  * Area load q = pressure + gamma t along -Z, consistent nodal values
//    f_a = -q sum_g N_a(g) detJ(g).
//
// Mapping: one thread per element.  A quad costs about 6,000 FP64 operations,
// once per design evaluation, and keeps GB300's FP64 pipe ~86 % busy; the
// solve (thousands of CG iterations) dominates every workload.
#include <math.h>

#include "sso_internal.cuh"

namespace sso {
namespace {

// Element kernels run one element per thread and are bound by the FP64 pipe
// (about 2 FP64 operations per clock per SM on GB300), so they are launched as
// 32-thread CTAs: a small model's few elements spread over many SMs instead
// of sharing the FP64 pipe of one (the 261 beams of the 10 x 10 grid-shell:
// 42 us in 128-thread CTAs).  A large batch keeps the same occupancy (the
// quad kernels' registers allow 8 such CTAs per SM).
constexpr int EL_THREADS = 32;

// ---------------------------------------------------------------------------
// Forward-mode dual number with N tangents (adjoint kernels).
template <int N>
struct DN {
  double v;
  double d[N];
  __device__ DN() {}
  __device__ DN(double a) : v(a) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
};
template <int N>
__device__ __forceinline__ DN<N> operator+(const DN<N>& a, const DN<N>& b) {
  DN<N> c;
  c.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) c.d[i] = a.d[i] + b.d[i];
  return c;
}
template <int N>
__device__ __forceinline__ DN<N> operator-(const DN<N>& a, const DN<N>& b) {
  DN<N> c;
  c.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) c.d[i] = a.d[i] - b.d[i];
  return c;
}
template <int N>
__device__ __forceinline__ DN<N> operator-(const DN<N>& a) {
  DN<N> c;
  c.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) c.d[i] = -a.d[i];
  return c;
}
template <int N>
__device__ __forceinline__ DN<N> operator*(const DN<N>& a, const DN<N>& b) {
  DN<N> c;
  c.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) c.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return c;
}
template <int N>
__device__ __forceinline__ DN<N> operator*(double a, const DN<N>& b) {
  DN<N> c;
  c.v = a * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) c.d[i] = a * b.d[i];
  return c;
}
template <int N>
__device__ __forceinline__ DN<N> operator*(const DN<N>& b, double a) {
  return a * b;
}
template <int N>
__device__ __forceinline__ DN<N> operator/(const DN<N>& a, const DN<N>& b) {
  DN<N> c;
  const double inv = 1.0 / b.v;
  c.v = a.v * inv;
#pragma unroll
  for (int i = 0; i < N; ++i) c.d[i] = (a.d[i] - c.v * b.d[i]) * inv;
  return c;
}
template <int N>
__device__ __forceinline__ DN<N> sqrt(const DN<N>& a) {
  DN<N> c;
  c.v = ::sqrt(a.v);
  const double h = 0.5 / c.v;
#pragma unroll
  for (int i = 0; i < N; ++i) c.d[i] = a.d[i] * h;
  return c;
}
__device__ __forceinline__ double sqrt(double a) { return ::sqrt(a); }
__device__ __forceinline__ double value(double a) { return a; }
template <int N>
__device__ __forceinline__ double value(const DN<N>& a) { return a.v; }

template <class S>
__device__ __forceinline__ void cross(const S a[3], const S b[3], S c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
template <class S>
__device__ __forceinline__ S dot(const S a[3], const S b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// ---------------------------------------------------------------------------
// Quad geometry.
constexpr double GP = 0.57735026918962576451;  // 1/sqrt(3)
__device__ __constant__ double kXiN[4] = {-1.0, 1.0, 1.0, -1.0};
__device__ __constant__ double kEtaN[4] = {-1.0, -1.0, 1.0, 1.0};

template <class S>
struct QuadGeom {
  S R[3][3];  // rows: local x, local y, normal (global components)
  S x[4], y[4], h[4];
};

template <class S>
__device__ void quad_geom(const S X[4][3], QuadGeom<S>& g) {
  S c[3], d13[3], d24[3], nv[3], a[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c[k] = 0.25 * (X[0][k] + X[1][k] + X[2][k] + X[3][k]);
    d13[k] = X[2][k] - X[0][k];
    d24[k] = X[3][k] - X[1][k];
    a[k] = (X[1][k] - X[0][k]) + (X[2][k] - X[3][k]);
  }
  cross(d13, d24, nv);
  const S inv_n = S(1.0) / sqrt(dot(nv, nv));
  S n[3] = {nv[0] * inv_n, nv[1] * inv_n, nv[2] * inv_n};
  const S an = dot(a, n);
#pragma unroll
  for (int k = 0; k < 3; ++k) a[k] = a[k] - an * n[k];
  const S inv_a = S(1.0) / sqrt(dot(a, a));
  S e1[3] = {a[0] * inv_a, a[1] * inv_a, a[2] * inv_a};
  S e2[3];
  cross(n, e1, e2);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    g.R[0][k] = e1[k];
    g.R[1][k] = e2[k];
    g.R[2][k] = n[k];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    S r[3] = {X[i][0] - c[0], X[i][1] - c[1], X[i][2] - c[2]};
    g.x[i] = dot(r, e1);
    g.y[i] = dot(r, e2);
    g.h[i] = dot(r, n);
  }
}

// Shape functions, their natural derivatives and the facet Jacobian.
template <class S>
struct QuadPoint {
  double N[4], Nxi[4], Neta[4];
  S xxi, yxi, xeta, yeta;
};

template <class S>
__device__ void quad_point(const QuadGeom<S>& g, double xi, double eta, QuadPoint<S>& P) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    P.N[i] = 0.25 * (1.0 + kXiN[i] * xi) * (1.0 + kEtaN[i] * eta);
    P.Nxi[i] = 0.25 * kXiN[i] * (1.0 + kEtaN[i] * eta);
    P.Neta[i] = 0.25 * kEtaN[i] * (1.0 + kXiN[i] * xi);
  }
  P.xxi = P.Nxi[0] * g.x[0] + P.Nxi[1] * g.x[1] + P.Nxi[2] * g.x[2] + P.Nxi[3] * g.x[3];
  P.yxi = P.Nxi[0] * g.y[0] + P.Nxi[1] * g.y[1] + P.Nxi[2] * g.y[2] + P.Nxi[3] * g.y[3];
  P.xeta = P.Neta[0] * g.x[0] + P.Neta[1] * g.x[1] + P.Neta[2] * g.x[2] + P.Neta[3] * g.x[3];
  P.yeta = P.Neta[0] * g.y[0] + P.Neta[1] * g.y[1] + P.Neta[2] * g.y[2] + P.Neta[3] * g.y[3];
}

// Covariant transverse shear rows at a tying point, per node over (w, rx, ry):
// g_xi = w_xi + beta.x_xi and g_eta = w_eta + beta.x_eta, beta = (ry, -rx).
template <class S>
__device__ void tying_rows(const QuadGeom<S>& g, double xi, double eta, S gxi[4][3],
                           S geta[4][3]) {
  QuadPoint<S> P;
  quad_point(g, xi, eta, P);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    gxi[i][0] = S(P.Nxi[i]);
    gxi[i][1] = -P.N[i] * P.yxi;
    gxi[i][2] = P.N[i] * P.xxi;
    geta[i][0] = S(P.Neta[i]);
    geta[i][1] = -P.N[i] * P.yeta;
    geta[i][2] = P.N[i] * P.xeta;
  }
}

// Everything a Gauss point contributes: Cartesian shape derivatives, the area
// weight detJ and the assumed-strain shear rows Bs[c][node][(w, rx, ry)].
template <class S>
struct GaussData {
  double N[4];
  S Nx[4], Ny[4], detJ;
  S Bs[2][4][3];
};

template <class S>
__device__ void gauss_data(const QuadGeom<S>& g, int gi, int gj, const S tB[4][3],
                           const S tD[4][3], const S tA[4][3], const S tC[4][3],
                           GaussData<S>& G) {
  const double xi = gi == 0 ? -GP : GP;
  const double eta = gj == 0 ? -GP : GP;
  QuadPoint<S> P;
  quad_point(g, xi, eta, P);
  G.detJ = P.xxi * P.yeta - P.yxi * P.xeta;
  const S inv = S(1.0) / G.detJ;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    G.N[i] = P.N[i];
    G.Nx[i] = (P.yeta * P.Nxi[i] - P.yxi * P.Neta[i]) * inv;
    G.Ny[i] = (P.xxi * P.Neta[i] - P.xeta * P.Nxi[i]) * inv;
  }
  const double cB = 0.5 * (1.0 - eta), cD = 0.5 * (1.0 + eta);
  const double cA = 0.5 * (1.0 - xi), cC = 0.5 * (1.0 + xi);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const S gx = cB * tB[i][p] + cD * tD[i][p];
      const S ge = cA * tA[i][p] + cC * tC[i][p];
      G.Bs[0][i][p] = (P.yeta * gx - P.yxi * ge) * inv;
      G.Bs[1][i][p] = (P.xxi * ge - P.xeta * gx) * inv;
    }
}

struct QuadMaterial {
  double m11, m12, m22, m33;  // membrane D
  double b11, b12, b22, b33;  // bending D
  double ds, dd;              // shear, drilling
};

template <class S>
struct QuadMaterialT {
  S m11, m12, m22, m33, b11, b12, b22, b33, ds, dd;
};

template <class S>
__device__ void quad_material(S t, double E, double nu, double kx, double ky,
                              QuadMaterialT<S>& M) {
  const double G = E / (2.0 * (1.0 + nu));
  const double kxy = ::sqrt(kx * ky);
  const S cm = (E / (1.0 - nu * nu)) * t;
  const S cb = (E / (12.0 * (1.0 - nu * nu))) * (t * t * t);
  M.m11 = kx * cm;
  M.m22 = ky * cm;
  M.m12 = (nu * kxy) * cm;
  M.m33 = (kxy * (1.0 - nu) * 0.5) * cm;
  M.b11 = kx * cb;
  M.b22 = ky * cb;
  M.b12 = (nu * kxy) * cb;
  M.b33 = (kxy * (1.0 - nu) * 0.5) * cb;
  M.ds = (5.0 / 6.0 * G) * t;
  M.dd = (0.01 * G) * t;
}

// ---------------------------------------------------------------------------
// Element e's 16 node-pair blocks: block (a, b) goes to
// ke + 36 * pos(16 e + 4 a + b), pos = epos (assembly order) or the identity.
__device__ __forceinline__ void quad_stiffness_element(
    int e, const double* __restrict__ xyz, const int* __restrict__ conn,
    const double* __restrict__ props, double pressure, double gamma, double* __restrict__ ke,
    const int* __restrict__ epos, double* __restrict__ fslot) {
  double X[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int nd = conn[4 * e + a];
#pragma unroll
    for (int k = 0; k < 3; ++k) X[a][k] = xyz[3 * nd + k];
  }
  const double t = props[5 * e + 0], E = props[5 * e + 1], nu = props[5 * e + 2];
  const double kx = props[5 * e + 3], ky = props[5 * e + 4];

  QuadGeom<double> g;
  quad_geom(X, g);
  QuadMaterialT<double> M;
  quad_material<double>(t, E, nu, kx, ky, M);

  double tB[4][3], tD[4][3], tA[4][3], tC[4][3], dummy[4][3];
  tying_rows(g, 0.0, -1.0, tB, dummy);
  tying_rows(g, 0.0, 1.0, tD, dummy);
  tying_rows(g, -1.0, 0.0, dummy, tA);
  tying_rows(g, 1.0, 0.0, dummy, tC);

  GaussData<double> GD[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) gauss_data(g, k & 1, k >> 1, tB, tD, tA, tC, GD[k]);

  if (fslot) {
    const double q = pressure + gamma * t;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) s += GD[k].N[a] * GD[k].detJ;
      fslot[4 * e + a] = -q * s;
    }
  }

  auto block_out = [&](int a, int b) {
    const int eb = 16 * e + 4 * a + b;
    return ke + (size_t)(epos ? epos[eb] : eb) * 36;
  };
  for (int a = 0; a < 4; ++a) {
    for (int b = a; b < 4; ++b) {
      double K[6][6];
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) K[i][j] = 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const GaussData<double>& G = GD[k];
        const double w = G.detJ;
        const double xa = G.Nx[a], ya = G.Ny[a], xb = G.Nx[b], yb = G.Ny[b];
        // membrane (u, v)
        K[0][0] += w * (xa * M.m11 * xb + ya * M.m33 * yb);
        K[0][1] += w * (xa * M.m12 * yb + ya * M.m33 * xb);
        K[1][0] += w * (ya * M.m12 * xb + xa * M.m33 * yb);
        K[1][1] += w * (ya * M.m22 * yb + xa * M.m33 * xb);
        // bending (rx, ry): kappa = [ry_x, -rx_y, ry_y - rx_x]
        K[3][3] += w * (M.b22 * ya * yb + M.b33 * xa * xb);
        K[3][4] += w * (-M.b12 * ya * xb - M.b33 * xa * yb);
        K[4][3] += w * (-M.b12 * xa * yb - M.b33 * ya * xb);
        K[4][4] += w * (M.b11 * xa * xb + M.b33 * ya * yb);
        // assumed transverse shear (w, rx, ry)
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int r = 0; r < 3; ++r)
            K[2 + p][2 + r] +=
                w * M.ds * (G.Bs[0][a][p] * G.Bs[0][b][r] + G.Bs[1][a][p] * G.Bs[1][b][r]);
        // drilling (u, v, rz)
        const double da[3] = {0.5 * ya, -0.5 * xa, G.N[a]};
        const double db[3] = {0.5 * yb, -0.5 * xb, G.N[b]};
        const int id[3] = {0, 1, 5};
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int r = 0; r < 3; ++r) K[id[p]][id[r]] += w * M.dd * da[p] * db[r];
      }
      // rigid links to the mean plane: K <- W_a^T K W_b
      const double ha = g.h[a], hb = g.h[b];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        K[i][3] += hb * K[i][1];
        K[i][4] -= hb * K[i][0];
      }
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        K[3][j] += ha * K[1][j];
        K[4][j] -= ha * K[0][j];
      }
      // local -> global: each 3x3 sub-block M -> R^T M R
      double Kg[6][6];
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          double T[3][3];
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
              T[i][j] = K[3 * p + i][3 * r + 0] * g.R[0][j] + K[3 * p + i][3 * r + 1] * g.R[1][j] +
                        K[3 * p + i][3 * r + 2] * g.R[2][j];
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
              Kg[3 * p + i][3 * r + j] =
                  g.R[0][i] * T[0][j] + g.R[1][i] * T[1][j] + g.R[2][i] * T[2][j];
        }
      double* oab = block_out(a, b);
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) oab[i * 6 + j] = Kg[i][j];
      if (a != b) {
        double* oba = block_out(b, a);
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
          for (int j = 0; j < 6; ++j) oba[j * 6 + i] = Kg[i][j];
      }
    }
  }
}

__global__ void __launch_bounds__(128) quad_stiffness_kernel(
    int nq, const double* __restrict__ xyz, const int* __restrict__ conn,
    const double* __restrict__ props, double pressure, double gamma, double* __restrict__ ke,
    double* __restrict__ fslot) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nq) quad_stiffness_element(e, xyz, conn, props, pressure, gamma, ke, nullptr, fslot);
}

// Set-up stage of a batch: quads of job blockIdx.y, blocks in assembly order.
__global__ void __launch_bounds__(128) quad_setup_kernel(const SetupJob* __restrict__ jobs) {
  const SetupJob& J = jobs[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= J.n_quads) return;
  quad_stiffness_element(e, J.xyz, J.quad_conn, J.quad_props, J.pressure, J.gamma, J.kes,
                         J.epos + 4 * (size_t)J.n_beams, J.fslot + 2 * (size_t)J.n_beams);
}

// ---------------------------------------------------------------------------
// Beam-column.
template <class S>
__device__ void beam_frame(const S xi[3], const S xj[3], S R[3][3], S& L) {
  S d[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
  L = sqrt(dot(d, d));
  const S inv = S(1.0) / L;
  S ex[3] = {d[0] * inv, d[1] * inv, d[2] * inv};
  S ey[3], ez[3];
  if (fabs(value(ex[2])) > 1.0 - 1e-8) {
    ey[0] = S(0.0);
    ey[1] = S(1.0);
    ey[2] = S(0.0);
  } else {
    const S hx = -ex[1], hy = ex[0];
    const S hinv = S(1.0) / sqrt(hx * hx + hy * hy);
    ey[0] = hx * hinv;
    ey[1] = hy * hinv;
    ey[2] = S(0.0);
  }
  cross(ex, ey, ez);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    R[0][k] = ex[k];
    R[1][k] = ey[k];
    R[2][k] = ez[k];
  }
}

// Local 12x12 Euler-Bernoulli frame stiffness, dense.
__device__ void beam_local(double L, const double* p, double k[12][12]) {
  const double E = p[0], G = p[1], Iy = p[2], Iz = p[3], J = p[4], A = p[5];
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) k[i][j] = 0.0;
  const double ka = E * A / L, kt = G * J / L;
  k[0][0] = k[6][6] = ka;
  k[0][6] = k[6][0] = -ka;
  k[3][3] = k[9][9] = kt;
  k[3][9] = k[9][3] = -kt;
  // (v, rz) with Iz at dofs 1, 5, 7, 11; (w, ry) with Iy at 2, 4, 8, 10 (ry sign flipped)
  const double L2 = L * L, L3 = L2 * L;
  for (int plane = 0; plane < 2; ++plane) {
    const double EI = E * (plane == 0 ? Iz : Iy);
    const double s = plane == 0 ? 1.0 : -1.0;  // sign of the rotation coupling
    const int v1 = plane == 0 ? 1 : 2, r1 = plane == 0 ? 5 : 4;
    const int v2 = v1 + 6, r2 = r1 + 6;
    const double a = 12.0 * EI / L3, b = 6.0 * EI / L2, c = 4.0 * EI / L, e = 2.0 * EI / L;
    k[v1][v1] = a;      k[v1][r1] = s * b;  k[v1][v2] = -a;     k[v1][r2] = s * b;
    k[r1][v1] = s * b;  k[r1][r1] = c;      k[r1][v2] = -s * b; k[r1][r2] = e;
    k[v2][v1] = -a;     k[v2][r1] = -s * b; k[v2][v2] = a;      k[v2][r2] = -s * b;
    k[r2][v1] = s * b;  k[r2][r1] = e;      k[r2][v2] = -s * b; k[r2][r2] = c;
  }
}

// Beam e's 4 node-pair blocks: block (a, b) goes to ke + 36 * pos(4 e + 2 a + b).
__device__ __forceinline__ void beam_stiffness_element(int e, const double* __restrict__ xyz,
                                                       const int* __restrict__ conn,
                                                       const double* __restrict__ props,
                                                       double* __restrict__ ke,
                                                       const int* __restrict__ epos) {
  const int ni = conn[2 * e], nj = conn[2 * e + 1];
  double xi[3], xj[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    xi[k] = xyz[3 * ni + k];
    xj[k] = xyz[3 * nj + k];
  }
  double R[3][3], L;
  beam_frame(xi, xj, R, L);
  double p[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = props[6 * e + k];
  double k[12][12];
  beam_local(L, p, k);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int eb = 4 * e + 2 * a + b;
      double* out = ke + (size_t)(epos ? epos[eb] : eb) * 36;
      for (int p3 = 0; p3 < 2; ++p3)
        for (int r3 = 0; r3 < 2; ++r3) {
          const int i0 = 6 * a + 3 * p3, j0 = 6 * b + 3 * r3;
          double T[3][3];
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
              T[i][j] = k[i0 + i][j0 + 0] * R[0][j] + k[i0 + i][j0 + 1] * R[1][j] +
                        k[i0 + i][j0 + 2] * R[2][j];
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
              out[(3 * p3 + i) * 6 + 3 * r3 + j] =
                  R[0][i] * T[0][j] + R[1][i] * T[1][j] + R[2][i] * T[2][j];
        }
    }
}

__global__ void __launch_bounds__(128) beam_stiffness_kernel(
    int nb, const double* __restrict__ xyz, const int* __restrict__ conn,
    const double* __restrict__ props, double* __restrict__ ke) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nb) beam_stiffness_element(e, xyz, conn, props, ke, nullptr);
}

__global__ void __launch_bounds__(128) beam_setup_kernel(const SetupJob* __restrict__ jobs) {
  const SetupJob& J = jobs[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < J.n_beams) beam_stiffness_element(e, J.xyz, J.beam_conn, J.beam_props, J.kes, J.epos);
}

__global__ void store_setup_job_kernel(SetupJob* dst, const SetupJob job) { *dst = job; }

// ---------------------------------------------------------------------------
// Adjoint contractions (Eq. 6).  For every element the scalar
//   G(p) = -lambda_e^T k_e(p) u_e + mu_e^T f_e(p),  mu = lambda + w u,
// is evaluated with dual numbers whose tangents are the element's design
// variables (z of each node; thickness for quads); dG/dp is the element's
// share of dJ/dp.  lambda^T k_e u is the FEM bilinear form, computed from the
// strains of u and lambda at the Gauss points rather than from k_e itself.

__global__ void __launch_bounds__(128) quad_adjoint_kernel(
    int nq, const double* __restrict__ xyz, const int* __restrict__ conn,
    const double* __restrict__ props, double pressure, double gamma,
    const double* __restrict__ u, const double* __restrict__ lam, double lam_scale, double w,
    double* __restrict__ gslot, double* __restrict__ dt, const double* __restrict__ rho,
    double penal, double* __restrict__ drho) {
  typedef DN<5> D;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nq) return;
  int nd[4];
  D X[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    nd[a] = conn[4 * e + a];
#pragma unroll
    for (int k = 0; k < 3; ++k) X[a][k] = D(xyz[3 * nd[a] + k]);
    X[a][2].d[a] = 1.0;
  }
  D t(props[5 * e + 0]);
  t.d[4] = 1.0;
  const double E = props[5 * e + 1], nu = props[5 * e + 2];
  const double kx = props[5 * e + 3], ky = props[5 * e + 4];

  QuadGeom<D> g;
  quad_geom(X, g);
  QuadMaterialT<D> M;
  quad_material<D>(t, E, nu, kx, ky, M);

  // local (projected) DOFs of u and lambda: rotate, then apply the rigid links
  D ul[4][6], ll[4][6];
  double muz[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double ug[6], lg[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      ug[k] = u[6 * nd[a] + k];
      lg[k] = lam_scale * lam[6 * nd[a] + k];
    }
    muz[a] = lg[2] + w * ug[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      ul[a][i] = g.R[i][0] * ug[0] + g.R[i][1] * ug[1] + g.R[i][2] * ug[2];
      ul[a][3 + i] = g.R[i][0] * ug[3] + g.R[i][1] * ug[4] + g.R[i][2] * ug[5];
      ll[a][i] = g.R[i][0] * lg[0] + g.R[i][1] * lg[1] + g.R[i][2] * lg[2];
      ll[a][3 + i] = g.R[i][0] * lg[3] + g.R[i][1] * lg[4] + g.R[i][2] * lg[5];
    }
    ul[a][0] = ul[a][0] - g.h[a] * ul[a][4];
    ul[a][1] = ul[a][1] + g.h[a] * ul[a][3];
    ll[a][0] = ll[a][0] - g.h[a] * ll[a][4];
    ll[a][1] = ll[a][1] + g.h[a] * ll[a][3];
  }

  D tB[4][3], tD[4][3], tA[4][3], tC[4][3], dummy[4][3];
  tying_rows(g, 0.0, -1.0, tB, dummy);
  tying_rows(g, 0.0, 1.0, tD, dummy);
  tying_rows(g, -1.0, 0.0, dummy, tA);
  tying_rows(g, 1.0, 0.0, dummy, tC);

  const D q = D(pressure) + gamma * t;
  D energy(0.0), load(0.0);
#pragma unroll 1
  for (int k = 0; k < 4; ++k) {
    GaussData<D> G;
    gauss_data(g, k & 1, k >> 1, tB, tD, tA, tC, G);
    D eu[3] = {D(0.0), D(0.0), D(0.0)}, el[3] = {D(0.0), D(0.0), D(0.0)};
    D ku[3] = {D(0.0), D(0.0), D(0.0)}, kl[3] = {D(0.0), D(0.0), D(0.0)};
    D su[2] = {D(0.0), D(0.0)}, sl[2] = {D(0.0), D(0.0)};
    D du(0.0), dl(0.0);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      eu[0] = eu[0] + G.Nx[a] * ul[a][0];
      eu[1] = eu[1] + G.Ny[a] * ul[a][1];
      eu[2] = eu[2] + G.Ny[a] * ul[a][0] + G.Nx[a] * ul[a][1];
      el[0] = el[0] + G.Nx[a] * ll[a][0];
      el[1] = el[1] + G.Ny[a] * ll[a][1];
      el[2] = el[2] + G.Ny[a] * ll[a][0] + G.Nx[a] * ll[a][1];
      ku[0] = ku[0] + G.Nx[a] * ul[a][4];
      ku[1] = ku[1] - G.Ny[a] * ul[a][3];
      ku[2] = ku[2] + G.Ny[a] * ul[a][4] - G.Nx[a] * ul[a][3];
      kl[0] = kl[0] + G.Nx[a] * ll[a][4];
      kl[1] = kl[1] - G.Ny[a] * ll[a][3];
      kl[2] = kl[2] + G.Ny[a] * ll[a][4] - G.Nx[a] * ll[a][3];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        su[c] = su[c] + G.Bs[c][a][0] * ul[a][2] + G.Bs[c][a][1] * ul[a][3] +
                G.Bs[c][a][2] * ul[a][4];
        sl[c] = sl[c] + G.Bs[c][a][0] * ll[a][2] + G.Bs[c][a][1] * ll[a][3] +
                G.Bs[c][a][2] * ll[a][4];
      }
      du = du + 0.5 * G.Ny[a] * ul[a][0] - 0.5 * G.Nx[a] * ul[a][1] + G.N[a] * ul[a][5];
      dl = dl + 0.5 * G.Ny[a] * ll[a][0] - 0.5 * G.Nx[a] * ll[a][1] + G.N[a] * ll[a][5];
    }
    D em = el[0] * (M.m11 * eu[0] + M.m12 * eu[1]) + el[1] * (M.m12 * eu[0] + M.m22 * eu[1]) +
           el[2] * (M.m33 * eu[2]);
    D eb = kl[0] * (M.b11 * ku[0] + M.b12 * ku[1]) + kl[1] * (M.b12 * ku[0] + M.b22 * ku[1]) +
           kl[2] * (M.b33 * ku[2]);
    D es = M.ds * (sl[0] * su[0] + sl[1] * su[1]);
    D ed = M.dd * (dl * du);
    energy = energy + G.detJ * (em + eb + es + ed);
    D nsum = (G.N[0] * muz[0] + G.N[1] * muz[1] + G.N[2] * muz[2] + G.N[3] * muz[3]) * G.detJ;
    load = load + nsum;
  }
  const D Gt = load * (-q) - energy;
  if (gslot) {
#pragma unroll
    for (int a = 0; a < 4; ++a) gslot[4 * e + a] = Gt.d[a];
  }
  if (dt) dt[e] = Gt.d[4];
  // SIMP (Eq. simp_eq): E = rho^P E*, and k_e is linear in E, so
  // d(lambda^T k_e u)/d rho = (P / rho) lambda^T k_e u
  if (drho) drho[e] = -(penal / rho[e]) * energy.v;
}

__global__ void __launch_bounds__(128) beam_adjoint_kernel(
    int nb, const double* __restrict__ xyz, const int* __restrict__ conn,
    const double* __restrict__ props, const double* __restrict__ u,
    const double* __restrict__ lam, double lam_scale, double* __restrict__ gslot) {
  typedef DN<2> D;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nb) return;
  const int n[2] = {conn[2 * e], conn[2 * e + 1]};
  D xi[3], xj[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    xi[k] = D(xyz[3 * n[0] + k]);
    xj[k] = D(xyz[3 * n[1] + k]);
  }
  xi[2].d[0] = 1.0;
  xj[2].d[1] = 1.0;
  D R[3][3], L;
  beam_frame(xi, xj, R, L);
  D ul[12], ll[12];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double* ug = u + 6 * n[a] + 3 * h;
        const double* lg = lam + 6 * n[a] + 3 * h;
        ul[6 * a + 3 * h + i] = R[i][0] * ug[0] + R[i][1] * ug[1] + R[i][2] * ug[2];
        ll[6 * a + 3 * h + i] =
            lam_scale * (R[i][0] * lg[0] + R[i][1] * lg[1] + R[i][2] * lg[2]);
      }
  const double E = props[6 * e + 0], Gm = props[6 * e + 1], Iy = props[6 * e + 2];
  const double Iz = props[6 * e + 3], J = props[6 * e + 4], A = props[6 * e + 5];
  const D invL = D(1.0) / L;
  const D invL2 = invL * invL, invL3 = invL2 * invL;
  // axial and torsion: k (a1 - a2)(b1 - b2)
  D en = (E * A) * invL * ((ll[0] - ll[6]) * (ul[0] - ul[6]));
  en = en + (Gm * J) * invL * ((ll[3] - ll[9]) * (ul[3] - ul[9]));
  // bending: 4x4 forms on (v1, r1, v2, r2)
  for (int plane = 0; plane < 2; ++plane) {
    const double EI = E * (plane == 0 ? Iz : Iy);
    const double s = plane == 0 ? 1.0 : -1.0;
    const int v1 = plane == 0 ? 1 : 2, r1 = plane == 0 ? 5 : 4;
    const int v2 = v1 + 6, r2 = r1 + 6;
    const D a = (12.0 * EI) * invL3, b = (6.0 * s * EI) * invL2;
    const D c = (4.0 * EI) * invL, d = (2.0 * EI) * invL;
    const D lv = ll[v1] - ll[v2], uv = ul[v1] - ul[v2];
    // a lv uv + b [lv (r1+r2)_u + (r1+r2)_l uv] + c (l_r1 u_r1 + l_r2 u_r2) + d (l_r1 u_r2 + l_r2 u_r1)
    en = en + a * (lv * uv) + b * (lv * (ul[r1] + ul[r2]) + (ll[r1] + ll[r2]) * uv) +
         c * (ll[r1] * ul[r1] + ll[r2] * ul[r2]) + d * (ll[r1] * ul[r2] + ll[r2] * ul[r1]);
  }
  gslot[2 * e + 0] = -en.d[0];
  gslot[2 * e + 1] = -en.d[1];
}

// Material volume of the quads (Sec. 3.3): per quad the facet area A_e (the
// 2 x 2 Gauss integral of the facet Jacobian, as for the area loads) with its
// tangents along the z of its four nodes (dual numbers, one per node).
// vol[e] = A_e t_e, dt[e] = A_e, vslot[4e + a] = t_e dA_e / dz_a.
__global__ void __launch_bounds__(128) quad_volume_kernel(
    int nq, const double* __restrict__ xyz, const int* __restrict__ conn,
    const double* __restrict__ props, double* __restrict__ vslot, double* __restrict__ dt,
    double* __restrict__ vol) {
  typedef DN<4> D;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nq) return;
  D X[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int nd = conn[4 * e + a];
#pragma unroll
    for (int k = 0; k < 3; ++k) X[a][k] = D(xyz[3 * nd + k]);
    X[a][2].d[a] = 1.0;
  }
  QuadGeom<D> g;
  quad_geom(X, g);
  D A(0.0);
#pragma unroll
  for (int gj = 0; gj < 2; ++gj)
#pragma unroll
    for (int gi = 0; gi < 2; ++gi) {
      QuadPoint<D> P;
      quad_point(g, gi == 0 ? -GP : GP, gj == 0 ? -GP : GP, P);
      A = A + (P.xxi * P.yeta - P.yxi * P.xeta);
    }
  const double t = props[5 * e + 0];
  dt[e] = A.v;
  vol[e] = A.v * t;
#pragma unroll
  for (int a = 0; a < 4; ++a) vslot[4 * e + a] = t * A.d[a];
}

// out = sum of v[0..n) in a fixed order (one CTA: strided partial sums, then a
// fixed-shape tree), so the result does not depend on timing.
__global__ void __launch_bounds__(256) ordered_sum_kernel(int n, const double* __restrict__ v,
                                                          double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

cudaError_t launch_quad_volume(int n_quads, const double* xyz, const int* conn,
                               const double* props, double* vslot, double* dt, double* vol,
                               cudaStream_t s) {
  if (n_quads <= 0) return cudaSuccess;
  quad_volume_kernel<<<(n_quads + EL_THREADS - 1) / EL_THREADS, EL_THREADS, 0, s>>>(n_quads, xyz, conn, props, vslot,
                                                            dt, vol);
  return cudaGetLastError();
}

cudaError_t launch_ordered_sum(int n, const double* v, double* out, cudaStream_t s) {
  ordered_sum_kernel<<<1, 256, 0, s>>>(n, v, out);
  return cudaGetLastError();
}

cudaError_t launch_beam_stiffness(int n_beams, const double* xyz, const int* conn,
                                  const double* props, double* ke, cudaStream_t s) {
  if (n_beams <= 0) return cudaSuccess;
  beam_stiffness_kernel<<<(n_beams + EL_THREADS - 1) / EL_THREADS, EL_THREADS, 0, s>>>(n_beams, xyz, conn, props, ke);
  return cudaGetLastError();
}

cudaError_t launch_store_setup_job(SetupJob* dst, const SetupJob& job, cudaStream_t s) {
  store_setup_job_kernel<<<1, 1, 0, s>>>(dst, job);
  return cudaGetLastError();
}

cudaError_t launch_setup_beams(const SetupJob* jobs, int n_jobs, int max_beams, cudaStream_t s) {
  if (n_jobs <= 0 || max_beams <= 0) return cudaSuccess;
  if (n_jobs > 65535) return cudaErrorInvalidValue;
  beam_setup_kernel<<<dim3((max_beams + EL_THREADS - 1) / EL_THREADS, n_jobs), EL_THREADS, 0, s>>>(jobs);
  return cudaGetLastError();
}

cudaError_t launch_setup_quads(const SetupJob* jobs, int n_jobs, int max_quads, cudaStream_t s) {
  if (n_jobs <= 0 || max_quads <= 0) return cudaSuccess;
  if (n_jobs > 65535) return cudaErrorInvalidValue;
  quad_setup_kernel<<<dim3((max_quads + EL_THREADS - 1) / EL_THREADS, n_jobs), EL_THREADS, 0, s>>>(jobs);
  return cudaGetLastError();
}

cudaError_t launch_quad_stiffness(int n_quads, const double* xyz, const int* conn,
                                  const double* props, double pressure, double gamma,
                                  double* ke, double* fslot, cudaStream_t s) {
  if (n_quads <= 0) return cudaSuccess;
  quad_stiffness_kernel<<<(n_quads + EL_THREADS - 1) / EL_THREADS, EL_THREADS, 0, s>>>(n_quads, xyz, conn, props,
                                                               pressure, gamma, ke, fslot);
  return cudaGetLastError();
}

cudaError_t launch_beam_adjoint(int n_beams, const double* xyz, const int* conn,
                                const double* props, const double* u, const double* lam,
                                double lam_scale, double* gslot, cudaStream_t s) {
  if (n_beams <= 0) return cudaSuccess;
  beam_adjoint_kernel<<<(n_beams + EL_THREADS - 1) / EL_THREADS, EL_THREADS, 0, s>>>(n_beams, xyz, conn, props, u, lam,
                                                             lam_scale, gslot);
  return cudaGetLastError();
}

cudaError_t launch_quad_adjoint(int n_quads, const double* xyz, const int* conn,
                                const double* props, double pressure, double gamma,
                                const double* u, const double* lam, double lam_scale,
                                double w, double* gslot, double* dt, cudaStream_t s,
                                const double* rho, double penal, double* drho) {
  if (n_quads <= 0) return cudaSuccess;
  quad_adjoint_kernel<<<(n_quads + EL_THREADS - 1) / EL_THREADS, EL_THREADS, 0, s>>>(
      n_quads, xyz, conn, props, pressure, gamma, u, lam, lam_scale, w, gslot, dt, rho, penal,
      drho);
  return cudaGetLastError();
}

// SIMP moduli (Eq. simp_eq): E_e = rho_e^P E*_e into the quads' properties.
__global__ void simp_kernel(int nq, const double* __restrict__ rho,
                            const double* __restrict__ E0, double penal,
                            double* __restrict__ props) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nq) props[5 * e + 1] = ::pow(rho[e], penal) * E0[e];
}

cudaError_t launch_simp(int n_quads, const double* rho, const double* E0, double penal,
                        double* props, cudaStream_t s) {
  if (n_quads <= 0) return cudaSuccess;
  simp_kernel<<<(n_quads + 127) / 128, 128, 0, s>>>(n_quads, rho, E0, penal, props);
  return cudaGetLastError();
}

}  // namespace sso
