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
// (N_f the face's unnormal normal, e_i the edge opposite i), gathered over the vertex's incidence
// list in face order (atomic-free). The solve is the PCG path of the smoothing step.
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
  const int e0 = md.incptr[v], e1 = md.incptr[v + 1];
  for (int e = e0; e < e1; ++e) {
    const int2 ic = md.inc[e];
    const int f = ic.x >> 2, c = ic.x & 3;
    double p[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int vid = md.F[3 * f + a];
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

}  // namespace ig
