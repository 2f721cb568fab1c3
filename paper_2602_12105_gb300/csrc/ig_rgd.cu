// ig_rgd.cu -- the u-step of the ADMM scheme for regularized geodesic distances (the geodesics
// application; formulation eq. edelstein): with per-face iterates y and z (the dual variable and
// the auxiliary z = G u),
//   b = m - D y + rho D z,    L u = b / (beta + rho) on the vertices that are not sources,
//   u = 0 on the sources,
// where m is the lumped vertex area, G the face gradient of piecewise-linear functions and
// D = G^T A_F its area-weighted adjoint (so that L = D G is the cotangent Laplacian).
//
// The operator: the mesh is assembled with t = 1 (A = M + L), and rgd_operator_kernel rewrites the
// values in place into the Laplacian with the sources' rows and columns replaced by the identity
// (so the sources decouple and stay 0), with the new Jacobi diagonal. The right-hand side:
//   (D w)_i = sum over the faces f at i of area_f <grad phi_i, w_f> = sum_f <N_f x e_i, w_f> / (2 |N_f|)
// (N_f the face's unnormalized normal, e_i the edge opposite i), gathered over the vertex's incidence
// list in face order (atomic-free). The solve is the PCG path of the smoothing step.
//
// Gradients (for gu = dl/du): lam = L_D^-1 gu (L_D the constrained operator, lam = 0 on sources),
//   dl/dy_f = -s area_f grad(lam)_f,  dl/dz_f = rho s area_f grad(lam)_f   (s = 1 / (beta + rho)),
//   dl/dV = s <lam, dm> - <lam, dL u> + s <lam, dD (rho z - y)>.
// The first two terms are the smoothing step's VJP with t = 1 (A = M + L), B = u + s and U = u;
// the last: per face, sum_c lam_c area <grad phi_c, W> = n . (E x W) / 2 with E = sum_c lam_c e_c,
// differentiated through E (linear in the positions) and the unit normal n.
//
// The ADMM rounds around the u-step (rgd_zy_kernel, per face): g = G u = N x (sum_c u_c e_c) / |N|^2,
// z = P(y / rho + g) with P the projection onto the unit ball, y += rho (beta_k g + (1 - beta_k)
// z_old - z); the primal residual max_f |g - z| is kept as a maximum over faces (exact, so free of
// the order of the faces).
//
// The fixed-point adjoint of the rounds (the implicit layer of the framework's fixed-point
// interface, for the geodesics application): at a fixed point x* = (y*, z*) = T(x*) of one round
// T, dl/dV = gV0 + (dT/dV)^T w with (I - J^T) w = (gy0, gz0), J = dT/dx and (gV0, gy0, gz0) the
// u-step's VJP of gu. A product J^T w (w = (wy, wz)) follows the round's three steps backwards:
//   rgd_rvjp_face: abar = dP(a)^T (wz - rho wy) with a = y / rho + G u (dP = I inside the unit ball,
//     (I - ahat ahat^T) / |a| outside), gbar = rho beta_k wy + abar (the cotangent of G u), and the
//     face parts of (I - J^T) w: -abar / rho for y, wz - rho (1 - beta_k) wy for z;
//   rgd_gT: ubar = G^T gbar (0 on the sources), then lam = L_D^-1 ubar;
//   rgd_lamgrad: the u-step's part, area grad(lam) times -s for y and rho s for z (taken with the
//     opposite sign inside I - J^T).
// (dT/dV)^T w is the same chain with ubar += gu: the u-step's VJP of the sum, plus rgd_gdface, the
// derivative of <gbar, G u> at fixed u (G u = N x E / |N|^2 per face, through E and N).
#include "ig_device.cuh"

namespace ig {

namespace {

// One thread per row: L = A - M on the diagonal (t = 1), identity rows and columns at sources.
__global__ void __launch_bounds__(kBlock) rgd_operator_kernel(const MeshDev* __restrict__ mds,
                                                              const int* __restrict__ src) {
  const MeshDev& md = mds[0];
  const int v = blockIdx.x * kBlock + threadIdx.x;
  if (v >= md.n) return;
  const int r0 = md.rowptr[v];
  const int len = md.rowptr[v + 1] - r0;
  const int sbase = md.sell_ptr[v >> 5] + (v & 31);
  const bool sv = src[v] != 0;
  double diag = 1.0;
  for (int j = 0; j < len; ++j) {
    const int c = md.col[r0 + j];
    const long at = sbase + 32L * j;
    double a = md.A[at];
    if (sv) {
      a = (c == v) ? 1.0 : 0.0;
    } else if (c == v) {
      a -= md.M[v];
      diag = a;
    } else if (src[c] != 0) {
      a = 0.0;
    }
    md.A[at] = a;
  }
  md.Dinv[v] = 1.0 / diag;
}

// b_i = (m_i - (D (y - rho z))_i) / (beta + rho), and 0 at the sources.
__global__ void __launch_bounds__(kBlock) rgd_rhs_kernel(const MeshDev* __restrict__ mds,
                                                         const double* __restrict__ V, const double* __restrict__ y,
                                                         const double* __restrict__ z, double rho, double scale,
                                                         const int* __restrict__ src, double* __restrict__ b) {
  const MeshDev& md = mds[0];
  const int v = blockIdx.x * kBlock + threadIdx.x;
  if (v >= md.n) return;
  if (src[v] != 0) {
    b[v] = 0.0;
    return;
  }
  double div = 0.0;
  int e0, e1;
  inc_range(md, v, e0, e1);
  for (int e = e0; e < e1; ++e) {
    const int2 ic = md.inc[e];
    const int f = inc_face(md, ic.x), c = ic.x & 3;
    double p[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int vid = face_vertex(md, f, a);
#pragma unroll
      for (int d = 0; d < 3; ++d) p[a][d] = V[3 * (long)vid + d];
    }
    double e1v[3], e2v[3], ec[3], N[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      e1v[d] = p[1][d] - p[0][d];
      e2v[d] = p[2][d] - p[0][d];
      ec[d] = p[(c + 2) % 3][d] - p[(c + 1) % 3][d];
    }
    N[0] = e1v[1] * e2v[2] - e1v[2] * e2v[1];
    N[1] = e1v[2] * e2v[0] - e1v[0] * e2v[2];
    N[2] = e1v[0] * e2v[1] - e1v[1] * e2v[0];
    const double inv2 = 0.5 / sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    double g[3];  // area_f * grad phi_c = N x e_c / (2 |N|)
    g[0] = (N[1] * ec[2] - N[2] * ec[1]) * inv2;
    g[1] = (N[2] * ec[0] - N[0] * ec[2]) * inv2;
    g[2] = (N[0] * ec[1] - N[1] * ec[0]) * inv2;
#pragma unroll
    for (int d = 0; d < 3; ++d) div = fma(g[d], y[3 * (long)f + d] - rho * z[3 * (long)f + d], div);
  }
  b[v] = (md.M[v] - div) * scale;
}

// gu with zeros on the sources (the adjoint right-hand side), or u + s (the VJP's B) when add_s.
__global__ void __launch_bounds__(kBlock) rgd_vec_kernel(const double* __restrict__ x, const int* __restrict__ src,
                                                         int n, int add_s, double s, double* __restrict__ out) {
  const int v = blockIdx.x * kBlock + threadIdx.x;
  if (v >= n) return;
  out[v] = add_s ? x[v] + s : (src[v] != 0 ? 0.0 : x[v]);
}

// Per face: the derivative of s * n . (E x W) / 2 (W = rho z - y) with respect to the corners,
// into gface [m][9]; and area grad(lam) = n x E / 2 for dl/dy and dl/dz.
__global__ void __launch_bounds__(kBlock) rgd_dface_kernel(const MeshDev* __restrict__ mds,
                                                           const double* __restrict__ V, const double* __restrict__ y,
                                                           const double* __restrict__ z, double rho, double s,
                                                           double* __restrict__ gy, double* __restrict__ gz) {
  const MeshDev& md = mds[0];
  const int f = blockIdx.x * kBlock + threadIdx.x;
  if (f >= md.m) return;
  double p[3][3], l[3];
  for (int c = 0; c < 3; ++c) {
    const int vid = face_vertex(md, f, c);
    l[c] = md.lam[vid];
    for (int d = 0; d < 3; ++d) p[c][d] = V[3 * (long)vid + d];
  }
  double a[3], b[3], N[3], E[3], W[3];
  for (int d = 0; d < 3; ++d) {
    a[d] = p[1][d] - p[0][d];
    b[d] = p[2][d] - p[0][d];
    // E = sum_c lam_c e_c, e_c = p_{c+2} - p_{c+1}
    E[d] = l[0] * (p[2][d] - p[1][d]) + l[1] * (p[0][d] - p[2][d]) + l[2] * (p[1][d] - p[0][d]);
    W[d] = rho * z[3 * (long)f + d] - y[3 * (long)f + d];
  }
  N[0] = a[1] * b[2] - a[2] * b[1];
  N[1] = a[2] * b[0] - a[0] * b[2];
  N[2] = a[0] * b[1] - a[1] * b[0];
  const double nN = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
  double n[3], wxn[3], exw[3], v[3], ga[3], gb[3];
  for (int d = 0; d < 3; ++d) n[d] = N[d] / nN;
  wxn[0] = W[1] * n[2] - W[2] * n[1];
  wxn[1] = W[2] * n[0] - W[0] * n[2];
  wxn[2] = W[0] * n[1] - W[1] * n[0];
  exw[0] = E[1] * W[2] - E[2] * W[1];
  exw[1] = E[2] * W[0] - E[0] * W[2];
  exw[2] = E[0] * W[1] - E[1] * W[0];
  const double en = exw[0] * n[0] + exw[1] * n[1] + exw[2] * n[2];
  for (int d = 0; d < 3; ++d) v[d] = (exw[d] - en * n[d]) / nN;
  ga[0] = b[1] * v[2] - b[2] * v[1];
  ga[1] = b[2] * v[0] - b[0] * v[2];
  ga[2] = b[0] * v[1] - b[1] * v[0];
  gb[0] = v[1] * a[2] - v[2] * a[1];
  gb[1] = v[2] * a[0] - v[0] * a[2];
  gb[2] = v[0] * a[1] - v[1] * a[0];
  double* out = md.gface + 9 * (long)f;
  for (int c = 0; c < 3; ++c) {
    const double dl = l[(c + 1) % 3] - l[(c + 2) % 3];
    for (int d = 0; d < 3; ++d) {
      double g = dl * wxn[d];
      if (c == 1) g += ga[d];
      else if (c == 2) g += gb[d];
      else g -= ga[d] + gb[d];
      out[3 * c + d] = 0.5 * s * g;
    }
  }
  if (gy || gz) {
    double ag[3];  // area grad(lam) = n x E / 2
    ag[0] = 0.5 * (n[1] * E[2] - n[2] * E[1]);
    ag[1] = 0.5 * (n[2] * E[0] - n[0] * E[2]);
    ag[2] = 0.5 * (n[0] * E[1] - n[1] * E[0]);
    for (int d = 0; d < 3; ++d) {
      if (gy) gy[3 * (long)f + d] = -s * ag[d];
      if (gz) gz[3 * (long)f + d] = rho * s * ag[d];
    }
  }
}

// gV[v] += sum over the faces at v (incidence order) of their corner's entry of gface.
__global__ void __launch_bounds__(kBlock) rgd_dgather_kernel(const MeshDev* __restrict__ mds, double* __restrict__ gV) {
  const MeshDev& md = mds[0];
  const int v = blockIdx.x * kBlock + threadIdx.x;
  if (v >= md.n) return;
  double g[3] = {0.0, 0.0, 0.0};
  int e0, e1;
  inc_range(md, v, e0, e1);
  for (int e = e0; e < e1; ++e) {
    const int2 ic = md.inc[e];
    const int f = inc_face(md, ic.x), c = ic.x & 3;
    for (int d = 0; d < 3; ++d) g[d] += md.gface[9 * (long)f + 3 * c + d];
  }
  for (int d = 0; d < 3; ++d) gV[3 * (long)v + d] += g[d];
}

// One z-step and dual step per face; primal (when not null) receives max_f |g - z| by atomicMax on
// the bits of a non-negative double (ordered like the values).
__global__ void __launch_bounds__(kBlock) rgd_zy_kernel(const MeshDev* __restrict__ mds, const double* __restrict__ V,
                                                        const double* __restrict__ u, double* __restrict__ y,
                                                        double* __restrict__ z, double rho, double beta_k,
                                                        unsigned long long* primal) {
  const MeshDev& md = mds[0];
  const int f = blockIdx.x * kBlock + threadIdx.x;
  if (f >= md.m) return;
  double p[3][3], uc[3];
  for (int c = 0; c < 3; ++c) {
    const int vid = face_vertex(md, f, c);
    uc[c] = u[vid];
    for (int d = 0; d < 3; ++d) p[c][d] = V[3 * (long)vid + d];
  }
  double a[3], b[3], E[3], N[3], g[3];
  for (int d = 0; d < 3; ++d) {
    a[d] = p[1][d] - p[0][d];
    b[d] = p[2][d] - p[0][d];
    E[d] = uc[0] * (p[2][d] - p[1][d]) + uc[1] * (p[0][d] - p[2][d]) + uc[2] * (p[1][d] - p[0][d]);
  }
  N[0] = a[1] * b[2] - a[2] * b[1];
  N[1] = a[2] * b[0] - a[0] * b[2];
  N[2] = a[0] * b[1] - a[1] * b[0];
  const double inv = 1.0 / (N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
  g[0] = (N[1] * E[2] - N[2] * E[1]) * inv;
  g[1] = (N[2] * E[0] - N[0] * E[2]) * inv;
  g[2] = (N[0] * E[1] - N[1] * E[0]) * inv;
  double yo[3], zo[3], zn[3];
  for (int d = 0; d < 3; ++d) {
    yo[d] = y[3 * (long)f + d];
    zo[d] = z[3 * (long)f + d];
    zn[d] = yo[d] / rho + g[d];
  }
  const double nz = sqrt(zn[0] * zn[0] + zn[1] * zn[1] + zn[2] * zn[2]);
  const double den = nz >= 1.0 ? nz : 1.0;
  double r2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    zn[d] = zn[d] / den;
    y[3 * (long)f + d] = yo[d] + rho * (beta_k * g[d] + (1.0 - beta_k) * zo[d] - zn[d]);
    z[3 * (long)f + d] = zn[d];
    r2 = fma(g[d] - zn[d], g[d] - zn[d], r2);
  }
  if (primal) atomicMax(primal, (unsigned long long)__double_as_longlong(sqrt(r2)));
}

// Dual residual of a round: rho max over the non-source vertices of |(D (z - z_old))_i| / m_i
// (area-normalised, in the units of the primal residual), by atomicMax on double bits.
__global__ void __launch_bounds__(kBlock) rgd_dual_kernel(const MeshDev* __restrict__ mds,
                                                          const double* __restrict__ V, const double* __restrict__ z,
                                                          const double* __restrict__ zold, const int* __restrict__ src,
                                                          double rho, unsigned long long* dual) {
  const MeshDev& md = mds[0];
  const int v = blockIdx.x * kBlock + threadIdx.x;
  if (v >= md.n || src[v] != 0) return;
  double div = 0.0;
  int e0, e1;
  inc_range(md, v, e0, e1);
  for (int e = e0; e < e1; ++e) {
    const int2 ic = md.inc[e];
    const int f = inc_face(md, ic.x), c = ic.x & 3;
    double p[3][3];
    for (int a = 0; a < 3; ++a) {
      const int vid = face_vertex(md, f, a);
      for (int d = 0; d < 3; ++d) p[a][d] = V[3 * (long)vid + d];
    }
    double e1v[3], e2v[3], ec[3], N[3];
    for (int d = 0; d < 3; ++d) {
      e1v[d] = p[1][d] - p[0][d];
      e2v[d] = p[2][d] - p[0][d];
      ec[d] = p[(c + 2) % 3][d] - p[(c + 1) % 3][d];
    }
    N[0] = e1v[1] * e2v[2] - e1v[2] * e2v[1];
    N[1] = e1v[2] * e2v[0] - e1v[0] * e2v[2];
    N[2] = e1v[0] * e2v[1] - e1v[1] * e2v[0];
    const double inv2 = 0.5 / sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    const double g0 = (N[1] * ec[2] - N[2] * ec[1]) * inv2;
    const double g1 = (N[2] * ec[0] - N[0] * ec[2]) * inv2;
    const double g2 = (N[0] * ec[1] - N[1] * ec[0]) * inv2;
    div = fma(g0, z[3 * (long)f + 0] - zold[3 * (long)f + 0], div);
    div = fma(g1, z[3 * (long)f + 1] - zold[3 * (long)f + 1], div);
    div = fma(g2, z[3 * (long)f + 2] - zold[3 * (long)f + 2], div);
  }
  const double r = rho * fabs(div) / md.M[v];
  atomicMax(dual, (unsigned long long)__double_as_longlong(r));
}

// Per face, the round's backward step through the z- and y-updates (see the file header): gbar =
// rho beta_k wy + abar, and, when out is given, out_y = -abar / rho, out_z = wz - rho (1 - beta_k) wy.
// w and out hold [wy (m x 3) | wz (m x 3)].
__global__ void __launch_bounds__(kBlock) rgd_rvjp_face_kernel(const MeshDev* __restrict__ mds,
                                                               const double* __restrict__ V,
                                                               const double* __restrict__ u,
                                                               const double* __restrict__ y,
                                                               const double* __restrict__ w, double rho, double beta_k,
                                                               double* __restrict__ gbar, double* __restrict__ out) {
  const MeshDev& md = mds[0];
  const int f = blockIdx.x * kBlock + threadIdx.x;
  if (f >= md.m) return;
  const long m3 = 3L * md.m;
  double p[3][3], uc[3];
  for (int c = 0; c < 3; ++c) {
    const int vid = face_vertex(md, f, c);
    uc[c] = u[vid];
    for (int d = 0; d < 3; ++d) p[c][d] = V[3 * (long)vid + d];
  }
  double a[3], b[3], E[3], N[3], av[3], wy[3], wz[3], zb[3];
  for (int d = 0; d < 3; ++d) {
    a[d] = p[1][d] - p[0][d];
    b[d] = p[2][d] - p[0][d];
    E[d] = uc[0] * (p[2][d] - p[1][d]) + uc[1] * (p[0][d] - p[2][d]) + uc[2] * (p[1][d] - p[0][d]);
  }
  N[0] = a[1] * b[2] - a[2] * b[1];
  N[1] = a[2] * b[0] - a[0] * b[2];
  N[2] = a[0] * b[1] - a[1] * b[0];
  const double inv = 1.0 / (N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
  av[0] = y[3 * (long)f + 0] / rho + (N[1] * E[2] - N[2] * E[1]) * inv;
  av[1] = y[3 * (long)f + 1] / rho + (N[2] * E[0] - N[0] * E[2]) * inv;
  av[2] = y[3 * (long)f + 2] / rho + (N[0] * E[1] - N[1] * E[0]) * inv;
  for (int d = 0; d < 3; ++d) {
    wy[d] = w[3 * (long)f + d];
    wz[d] = w[m3 + 3 * (long)f + d];
    zb[d] = wz[d] - rho * wy[d];
  }
  const double na = sqrt(av[0] * av[0] + av[1] * av[1] + av[2] * av[2]);
  if (na > 1.0) {
    // (I - ahat ahat^T) zb / |a|
    const double proj = (av[0] * zb[0] + av[1] * zb[1] + av[2] * zb[2]) / (na * na);
    for (int d = 0; d < 3; ++d) zb[d] = (zb[d] - proj * av[d]) / na;
  }
  for (int d = 0; d < 3; ++d) {
    gbar[3 * (long)f + d] = rho * beta_k * wy[d] + zb[d];
    if (out) {
      out[3 * (long)f + d] = -zb[d] / rho;
      out[m3 + 3 * (long)f + d] = wz[d] - rho * (1.0 - beta_k) * wy[d];
    }
  }
}

// ubar_i = (G^T gbar)_i (+ add_i) = sum over the faces at i of <grad phi_i, gbar_f>, grad phi_i =
// N_f x e_i / |N_f|^2; 0 at the sources.
__global__ void __launch_bounds__(kBlock) rgd_gT_kernel(const MeshDev* __restrict__ mds, const double* __restrict__ V,
                                                        const double* __restrict__ gbar, const double* __restrict__ add,
                                                        const int* __restrict__ src, double* __restrict__ ubar) {
  const MeshDev& md = mds[0];
  const int v = blockIdx.x * kBlock + threadIdx.x;
  if (v >= md.n) return;
  if (src[v] != 0) {
    ubar[v] = 0.0;
    return;
  }
  double acc = add ? add[v] : 0.0;
  int e0, e1;
  inc_range(md, v, e0, e1);
  for (int e = e0; e < e1; ++e) {
    const int2 ic = md.inc[e];
    const int f = inc_face(md, ic.x), c = ic.x & 3;
    double p[3][3];
    for (int a = 0; a < 3; ++a) {
      const int vid = face_vertex(md, f, a);
      for (int d = 0; d < 3; ++d) p[a][d] = V[3 * (long)vid + d];
    }
    double e1v[3], e2v[3], ec[3], N[3];
    for (int d = 0; d < 3; ++d) {
      e1v[d] = p[1][d] - p[0][d];
      e2v[d] = p[2][d] - p[0][d];
      ec[d] = p[(c + 2) % 3][d] - p[(c + 1) % 3][d];
    }
    N[0] = e1v[1] * e2v[2] - e1v[2] * e2v[1];
    N[1] = e1v[2] * e2v[0] - e1v[0] * e2v[2];
    N[2] = e1v[0] * e2v[1] - e1v[1] * e2v[0];
    const double inv = 1.0 / (N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    const double g0 = (N[1] * ec[2] - N[2] * ec[1]) * inv;
    const double g1 = (N[2] * ec[0] - N[0] * ec[2]) * inv;
    const double g2 = (N[0] * ec[1] - N[1] * ec[0]) * inv;
    acc = fma(g0, gbar[3 * (long)f + 0], acc);
    acc = fma(g1, gbar[3 * (long)f + 1], acc);
    acc = fma(g2, gbar[3 * (long)f + 2], acc);
  }
  ubar[v] = acc;
}

// out_y += cy area grad(lam), out_z += cz area grad(lam), area grad(lam) = n x E / 2 with
// E = sum_c lam_c e_c (lam in md.lam).
__global__ void __launch_bounds__(kBlock) rgd_lamgrad_kernel(const MeshDev* __restrict__ mds,
                                                             const double* __restrict__ V, double cy, double cz,
                                                             double* __restrict__ out) {
  const MeshDev& md = mds[0];
  const int f = blockIdx.x * kBlock + threadIdx.x;
  if (f >= md.m) return;
  const long m3 = 3L * md.m;
  double p[3][3], l[3];
  for (int c = 0; c < 3; ++c) {
    const int vid = face_vertex(md, f, c);
    l[c] = md.lam[vid];
    for (int d = 0; d < 3; ++d) p[c][d] = V[3 * (long)vid + d];
  }
  double a[3], b[3], N[3], E[3];
  for (int d = 0; d < 3; ++d) {
    a[d] = p[1][d] - p[0][d];
    b[d] = p[2][d] - p[0][d];
    E[d] = l[0] * (p[2][d] - p[1][d]) + l[1] * (p[0][d] - p[2][d]) + l[2] * (p[1][d] - p[0][d]);
  }
  N[0] = a[1] * b[2] - a[2] * b[1];
  N[1] = a[2] * b[0] - a[0] * b[2];
  N[2] = a[0] * b[1] - a[1] * b[0];
  const double h = 0.5 / sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
  double ag[3];
  ag[0] = (N[1] * E[2] - N[2] * E[1]) * h;
  ag[1] = (N[2] * E[0] - N[0] * E[2]) * h;
  ag[2] = (N[0] * E[1] - N[1] * E[0]) * h;
  for (int d = 0; d < 3; ++d) {
    out[3 * (long)f + d] += cy * ag[d];
    out[m3 + 3 * (long)f + d] += cz * ag[d];
  }
}

// Per face: the derivative of <W, G u> = N . (E x W) / |N|^2 (E = sum_c u_c e_c) with respect to
// the corners, into gface [m][9] (u and W held fixed).
__global__ void __launch_bounds__(kBlock) rgd_gdface_kernel(const MeshDev* __restrict__ mds,
                                                            const double* __restrict__ V, const double* __restrict__ u,
                                                            const double* __restrict__ W) {
  const MeshDev& md = mds[0];
  const int f = blockIdx.x * kBlock + threadIdx.x;
  if (f >= md.m) return;
  double p[3][3], uc[3];
  for (int c = 0; c < 3; ++c) {
    const int vid = face_vertex(md, f, c);
    uc[c] = u[vid];
    for (int d = 0; d < 3; ++d) p[c][d] = V[3 * (long)vid + d];
  }
  double a[3], b[3], N[3], E[3], w[3];
  for (int d = 0; d < 3; ++d) {
    a[d] = p[1][d] - p[0][d];
    b[d] = p[2][d] - p[0][d];
    E[d] = uc[0] * (p[2][d] - p[1][d]) + uc[1] * (p[0][d] - p[2][d]) + uc[2] * (p[1][d] - p[0][d]);
    w[d] = W[3 * (long)f + d];
  }
  N[0] = a[1] * b[2] - a[2] * b[1];
  N[1] = a[2] * b[0] - a[0] * b[2];
  N[2] = a[0] * b[1] - a[1] * b[0];
  const double inn = 1.0 / (N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
  double wxn[3], X[3], v[3], ga[3], gb[3];
  // through E: dE . (W x N) / |N|^2
  wxn[0] = (w[1] * N[2] - w[2] * N[1]) * inn;
  wxn[1] = (w[2] * N[0] - w[0] * N[2]) * inn;
  wxn[2] = (w[0] * N[1] - w[1] * N[0]) * inn;
  // through N: v = X / |N|^2 - 2 (N . X) N / |N|^4, X = E x W; v . dN = da . (b x v) + db . (v x a)
  X[0] = E[1] * w[2] - E[2] * w[1];
  X[1] = E[2] * w[0] - E[0] * w[2];
  X[2] = E[0] * w[1] - E[1] * w[0];
  const double sv = (N[0] * X[0] + N[1] * X[1] + N[2] * X[2]) * inn;
  for (int d = 0; d < 3; ++d) v[d] = (X[d] - 2.0 * sv * N[d]) * inn;
  ga[0] = b[1] * v[2] - b[2] * v[1];
  ga[1] = b[2] * v[0] - b[0] * v[2];
  ga[2] = b[0] * v[1] - b[1] * v[0];
  gb[0] = v[1] * a[2] - v[2] * a[1];
  gb[1] = v[2] * a[0] - v[0] * a[2];
  gb[2] = v[0] * a[1] - v[1] * a[0];
  double* out = md.gface + 9 * (long)f;
  for (int c = 0; c < 3; ++c) {
    const double du = uc[(c + 1) % 3] - uc[(c + 2) % 3];
    for (int d = 0; d < 3; ++d) {
      double g = du * wxn[d];
      if (c == 1) g += ga[d];
      else if (c == 2) g += gb[d];
      else g -= ga[d] + gb[d];
      out[3 * c + d] = g;
    }
  }
}

// Warm start of a u-step solve from the previous round's u: rhs = b - A u with the constrained
// operator (the solve then finds the correction), and ratio = |b| / |rhs|, so that solving the
// correction to a relative tolerance of tol * ratio leaves |b - A u| <= tol |b|, the criterion of
// a cold solve. Tiles of kTileRows rows, 4 per thread; deterministic sums (last CTA, tile order).
__global__ void __launch_bounds__(kBlock) rgd_warm_kernel(const MeshDev* __restrict__ mds, const double* __restrict__ b,
                                                          const double* __restrict__ u, double* __restrict__ rhs,
                                                          double* ratio) {
  __shared__ double sh[2 * kBlock];
  const MeshDev& md = mds[0];
  const long n = md.n;
  const int ntile = (int)((n + kTileRows - 1) / kTileRows);
  double acc[2] = {0.0, 0.0};
#pragma unroll
  for (int rr = 0; rr < kRowsPerThread; ++rr) {
    const long row = (long)blockIdx.x * kTileRows + rr * kBlock + threadIdx.x;
    if (row < n) {
      double au[1];
      row_product<1>(md, md.A, row, GatherAoS64<1>{u}, au);
      const double bb = b[row], r = bb - au[0];
      rhs[row] = r;
      acc[0] = fma(bb, bb, acc[0]);
      acc[1] = fma(r, r, acc[1]);
    }
  }
  if (reduce_tiles<2>(acc, md.part, blockIdx.x, ntile, &md.s->cnt[2], sh) && threadIdx.x == 0)
    *ratio = acc[1] > 0.0 ? sqrt(acc[0] / acc[1]) : 1e300;
}

__global__ void __launch_bounds__(kBlock) rgd_axpy_kernel(double* __restrict__ u, const double* __restrict__ d, long n) {
  const long i = (long)blockIdx.x * kBlock + threadIdx.x;
  if (i < n) u[i] += d[i];
}

// The worst status of the solves so far (codes grow with severity: 0 ok, NOT_CONVERGED, NONFINITE).
__global__ void rgd_note_status_kernel(const MeshDev* __restrict__ mds, int* worst) {
  const int st = mds[0].s->status;
  if (st > *worst) *worst = st;
}

}  // namespace

cudaError_t launch_rgd_operator(const MeshDev* mds, int n, const int* src, cudaStream_t st) {
  IG_PROF("rgd_operator", st);
  rgd_operator_kernel<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(mds, src);
  return cudaGetLastError();
}

cudaError_t launch_rgd_rhs(const MeshDev* mds, int n, const double* V, const double* y, const double* z, double rho,
                           double beta, const int* src, double* b, cudaStream_t st) {
  IG_PROF("rgd_rhs", st);
  rgd_rhs_kernel<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(mds, V, y, z, rho, 1.0 / (beta + rho), src, b);
  return cudaGetLastError();
}

cudaError_t launch_rgd_warm(const MeshDev* mds, long n, const double* b, const double* u, double* rhs, double* ratio,
                            cudaStream_t st) {
  IG_PROF("rgd_warm", st);
  rgd_warm_kernel<<<(unsigned)((n + kTileRows - 1) / kTileRows), kBlock, 0, st>>>(mds, b, u, rhs, ratio);
  return cudaGetLastError();
}

cudaError_t launch_rgd_axpy(double* u, const double* d, long n, cudaStream_t st) {
  rgd_axpy_kernel<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(u, d, n);
  return cudaGetLastError();
}

cudaError_t launch_rgd_note_status(const MeshDev* mds, int* worst, cudaStream_t st) {
  rgd_note_status_kernel<<<1, 1, 0, st>>>(mds, worst);
  return cudaGetLastError();
}

cudaError_t launch_rgd_vec(const double* x, const int* src, int n, int add_s, double s, double* out, cudaStream_t st) {
  rgd_vec_kernel<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(x, src, n, add_s, s, out);
  return cudaGetLastError();
}

cudaError_t launch_rgd_dD(const MeshDev* mds, int n, int m, const double* V, const double* y, const double* z,
                          double rho, double beta, double* gV, double* gy, double* gz, cudaStream_t st) {
  {
    IG_PROF("rgd_dface", st);
    rgd_dface_kernel<<<(m + kBlock - 1) / kBlock, kBlock, 0, st>>>(mds, V, y, z, rho, 1.0 / (beta + rho), gy, gz);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    IG_PROF("rgd_dgather", st);
    rgd_dgather_kernel<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(mds, gV);
  }
  return cudaGetLastError();
}

cudaError_t launch_rgd_zy(const MeshDev* mds, int m, const double* V, const double* u, double* y, double* z, double rho,
                          double beta_k, unsigned long long* primal, cudaStream_t st) {
  IG_PROF("rgd_zy", st);
  rgd_zy_kernel<<<(m + kBlock - 1) / kBlock, kBlock, 0, st>>>(mds, V, u, y, z, rho, beta_k, primal);
  return cudaGetLastError();
}

cudaError_t launch_rgd_dual(const MeshDev* mds, int n, const double* V, const double* z, const double* zold,
                            const int* src, double rho, unsigned long long* dual, cudaStream_t st) {
  IG_PROF("rgd_dual", st);
  rgd_dual_kernel<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(mds, V, z, zold, src, rho, dual);
  return cudaGetLastError();
}

cudaError_t launch_rgd_rvjp_face(const MeshDev* mds, int m, const double* V, const double* u, const double* y,
                                 const double* w, double rho, double beta_k, double* gbar, double* out,
                                 cudaStream_t st) {
  IG_PROF("rgd_rvjp_face", st);
  rgd_rvjp_face_kernel<<<(m + kBlock - 1) / kBlock, kBlock, 0, st>>>(mds, V, u, y, w, rho, beta_k, gbar, out);
  return cudaGetLastError();
}

cudaError_t launch_rgd_gT(const MeshDev* mds, int n, const double* V, const double* gbar, const double* add,
                          const int* src, double* ubar, cudaStream_t st) {
  IG_PROF("rgd_gT", st);
  rgd_gT_kernel<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(mds, V, gbar, add, src, ubar);
  return cudaGetLastError();
}

cudaError_t launch_rgd_lamgrad(const MeshDev* mds, int m, const double* V, double cy, double cz, double* out,
                               cudaStream_t st) {
  IG_PROF("rgd_lamgrad", st);
  rgd_lamgrad_kernel<<<(m + kBlock - 1) / kBlock, kBlock, 0, st>>>(mds, V, cy, cz, out);
  return cudaGetLastError();
}

cudaError_t launch_rgd_dG(const MeshDev* mds, int n, int m, const double* V, const double* u, const double* W,
                          double* gV, cudaStream_t st) {
  {
    IG_PROF("rgd_gdface", st);
    rgd_gdface_kernel<<<(m + kBlock - 1) / kBlock, kBlock, 0, st>>>(mds, V, u, W);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    IG_PROF("rgd_dgather", st);
    rgd_dgather_kernel<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(mds, gV);
  }
  return cudaGetLastError();
}

}  // namespace ig
