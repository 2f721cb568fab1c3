// ig_eigs.cu -- shift-invert subspace iteration for the lowest eigenpairs of the pencil (L, M):
// the forward half of the eigenvector fixed point of Eq. eigiter (§5),
//   f(A, B, U) = Q((A - sigma B)^-1 B U) - U = 0,
// here with A = L, B = M and the shift sigma = -1/t of the assembled smoothing operator, so that
// (L - sigma M)^-1 M = t (M + t L)^-1 M: a step is the smoothing solve (M + tL) Y = M U (done by
// the PCG path, k columns together) followed by Q. The constant t drops out in Q.
//
// Q (per step): the Gram matrix G = Y^T M Y (k x k, tile partials added in tile order), its
// Cholesky factor G = R^T R (R upper triangular, on one thread of the CTA that completes the sum)
// and U = Y R^-1: the M-orthonormal basis of Y's columns in Gram-Schmidt order.
// After the last step: the canonical sign of each column (its first entry, in vertex order,
// within a relative 1e-6 of the column's largest magnitude is made positive; column signs of the
// intermediate iterates do not change the final basis) and lambda_c = u_c^T L u_c, computed as
// (u_c^T A u_c - u_c^T M u_c) / t with the FP64 operator A = M + tL.
//
// The gradient through the fixed point (eig_vjp_*): with S = (M + tL)^-1 M (t drops out in Q)
// and U* = Q(S U*), the implicit-function rule gives w = gU + J^T w (J = df/dU at U*), solved by
// its Neumann series, then dl/dV = (df/dV)^T w. For Y = S U*, Y = Qraw R (Qraw = U* diag(s), s the
// canonical signs) and a cotangent w on U*: Qb = w diag(s), P = R^-1 Phi(Qraw^T Qb) R^-T (Phi: upper
// triangle, half diagonal), Ybar = Qb R^-T - M Y (P + P^T); then J^T w = M (M + tL)^-1 Ybar, and
// dl/dV = <Lambda, d(M U*)/dV - dA/dV Y> with Lambda = (M + tL)^-1 Ybar, plus the Gram matrix's mass
// term d(sum_i M_i w_i)/dV with w_i = -Y_i P Y_i^T.
//
// Every reduction is over tiles of kBlock rows; the CTA that completes it (a counter) adds the
// tile partials in tile order, so results do not depend on scheduling.
#include <climits>

#include "ig_device.cuh"

namespace ig {

namespace {

constexpr int kEigStride = 16;        // doubles per tile partial
constexpr double kSignBand = 1e-6;    // relative band below the largest magnitude for the sign rule

// Small results: R^-1 (k x k, row-major), column maxima, signs, eigenvalues, status word.
struct EigSmall {
  double rinv[kMaxK * kMaxK];
  double p[kMaxK * kMaxK];   // P of the gradient step (row-major)
  double colmax[kMaxK];
  double sign[kMaxK];
  double lambda[kMaxK];
  double rdiag[kMaxK];     // diagonal of R of the last step: about 1 / (1 + t lambda_c) near convergence
  double tol_ratio;        // min_c |M U_c| / |M U_c - A Y0_c| of the warm start
  int sign_row[kMaxK];
  int fail;        // 1 once a Gram matrix was not numerically positive definite (dependent or non-finite columns)
  unsigned cnt;    // last-CTA counter, reset by the CTA that completes each reduction
};

// Publish this CTA's partials (thread 0 holds them in v) and return true in the CTA that completes
// the reduction; every thread of that CTA then sees the partials of all tiles.
__device__ __forceinline__ bool eig_publish(EigSmall* sm, int ntile) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&sm->cnt, 1u);
    s_last = (prev == (unsigned)ntile - 1u);
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Sum of the NV partials over all tiles in tile order: thread j adds tiles j, j + kBlock, ...,
// then the CTA adds the threads' sums in thread order. Thread 0 receives the totals.
template <int NV>
__device__ __forceinline__ void eig_gather_sum(const double* __restrict__ part, int ntile, double (&v)[NV],
                                               double* sh) {
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.0;
  for (int b = threadIdx.x; b < ntile; b += kBlock)
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __ldcg(part + (long)b * kEigStride + i);
  block_sum<NV>(v, sh);
}

// Maximum (MIN = false) or minimum (MIN = true) of part[b * kEigStride + off + c] over the tiles,
// for c < K; thread 0 receives the results (max and min are exact, so the order is free).
template <int K, bool MIN>
__device__ __forceinline__ void eig_gather_ext(const double* __restrict__ part, int ntile, int off, double (&v)[K]) {
  __shared__ double sw[K][kBlock / 32];
#pragma unroll
  for (int c = 0; c < K; ++c) v[c] = MIN ? 1e300 : 0.0;
  for (int b = threadIdx.x; b < ntile; b += kBlock)
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const double x = __ldcg(part + (long)b * kEigStride + off + c);
      v[c] = MIN ? fmin(v[c], x) : fmax(v[c], x);
    }
#pragma unroll
  for (int c = 0; c < K; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double x = __shfl_xor_sync(0xffffffffu, v[c], o);
      v[c] = MIN ? fmin(v[c], x) : fmax(v[c], x);
    }
    if ((threadIdx.x & 31) == 0) sw[c][threadIdx.x >> 5] = v[c];
  }
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < K; ++c) {
      double m = sw[c][0];
      for (int w = 1; w < kBlock / 32; ++w) m = MIN ? fmin(m, sw[c][w]) : fmax(m, sw[c][w]);
      v[c] = m;
    }
}

// ---------------------------------------------------------------------------------------------
// G = Y^T M Y, then R^-1 of its Cholesky factor.
template <int K>
__global__ void __launch_bounds__(kBlock) eig_gram_kernel(const double* __restrict__ Y, const double* __restrict__ M,
                                                          long n, double* __restrict__ part, EigSmall* sm) {
  constexpr int NG = K * (K + 1) / 2;
  __shared__ double sh[NG * kBlock];
  const int ntile = (int)((n + kBlock - 1) / kBlock);
  const long row = (long)blockIdx.x * kBlock + threadIdx.x;
  double acc[NG];
#pragma unroll
  for (int i = 0; i < NG; ++i) acc[i] = 0.0;
  if (row < n) {
    double y[K];
#pragma unroll
    for (int c = 0; c < K; ++c) y[c] = Y[row * K + c];
    const double m = M[row];
    int i = 0;
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
      for (int b = a; b < K; ++b) acc[i++] = m * y[a] * y[b];
  }
  block_sum<NG>(acc, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < NG; ++i) part[(long)blockIdx.x * kEigStride + i] = acc[i];
  if (!eig_publish(sm, ntile)) return;
  double g[NG];
  eig_gather_sum<NG>(part, ntile, g, sh);
  if (threadIdx.x != 0) return;
  // Cholesky G = R^T R (R upper triangular), then R^-1 by back substitution
  double G[K][K], R[K][K], Ri[K][K];
  int i = 0;
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int b = a; b < K; ++b) {
      G[a][b] = g[i];
      G[b][a] = g[i];
      ++i;
    }
  int bad = 0;
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int b = 0; b < K; ++b) {
      R[a][b] = 0.0;
      Ri[a][b] = 0.0;
    }
#pragma unroll
  for (int a = 0; a < K; ++a) {
    double d = G[a][a];
#pragma unroll
    for (int p = 0; p < a; ++p) d -= R[p][a] * R[p][a];
    // a pivot within rounding of zero relative to the column's own norm: the column depends on
    // the ones before it (exactly dependent columns leave a pivot of about 1e-16 G_aa)
    if (!(d > 1e-14 * G[a][a]) || !(d < 1e300)) {
      bad = 1;
      d = 1.0;
    }
    R[a][a] = sqrt(d);
#pragma unroll
    for (int b = a + 1; b < K; ++b) {
      double e = G[a][b];
#pragma unroll
      for (int p = 0; p < a; ++p) e -= R[p][a] * R[p][b];
      R[a][b] = e / R[a][a];
    }
  }
  // R^-1, column by column: R Ri[:, c] = e_c
#pragma unroll
  for (int c = 0; c < K; ++c) {
#pragma unroll
    for (int a = K - 1; a >= 0; --a) {
      double e = (a == c) ? 1.0 : 0.0;
#pragma unroll
      for (int p = a + 1; p < K; ++p) e -= R[a][p] * Ri[p][c];
      Ri[a][c] = e / R[a][a];
    }
  }
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int c = 0; c < K; ++c) sm->rinv[a * K + c] = Ri[a][c];
#pragma unroll
  for (int a = 0; a < K; ++a) sm->rdiag[a] = R[a][a];
  if (bad) sm->fail = 1;
  sm->cnt = 0u;
}

// Warm start of the next solve (A Y = M U): Y0 = U diag(rdiag), which A maps to about M U once U
// holds eigenvectors (A u = (1 + t lambda) M u); the solve then finds the correction from
// rhs = M U - A Y0, to a tolerance relative to |M U| rather than to |rhs| (tol_ratio).
template <int K>
__global__ void __launch_bounds__(kBlock) eig_warm_kernel(const MeshDev* __restrict__ mds,
                                                          const double* __restrict__ U, double* __restrict__ Y0,
                                                          double* __restrict__ rhs, double* __restrict__ part,
                                                          EigSmall* sm) {
  __shared__ double sh[2 * K * kBlock];
  __shared__ double rd[K];
  if (threadIdx.x < K) rd[threadIdx.x] = sm->rdiag[threadIdx.x];
  __syncthreads();
  const MeshDev& md = mds[0];
  const long n = md.n;
  const int ntile = (int)((n + kBlock - 1) / kBlock);
  const long row = (long)blockIdx.x * kBlock + threadIdx.x;
  double acc[2 * K];
#pragma unroll
  for (int i = 0; i < 2 * K; ++i) acc[i] = 0.0;
  if (row < n) {
    double au[K];
    row_product<K>(md, md.A, row, GatherAoS64<K>{U}, au);
    const double m = md.M[row];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const double u = U[row * K + c];
      const double mu = m * u;
      const double res = fma(-rd[c], au[c], mu);
      Y0[row * K + c] = rd[c] * u;
      rhs[row * K + c] = res;
      acc[c] = mu * mu;
      acc[K + c] = res * res;
    }
  }
  block_sum<2 * K>(acc, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) part[(long)blockIdx.x * kEigStride + i] = acc[i];
  if (!eig_publish(sm, ntile)) return;
  double tot[2 * K];
  eig_gather_sum<2 * K>(part, ntile, tot, sh);
  if (threadIdx.x == 0) {
    double ratio = 1e300;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const double rr = tot[K + c] > 0.0 ? sqrt(tot[c] / tot[K + c]) : 1e300;
      ratio = rr < ratio ? rr : ratio;
    }
    sm->tol_ratio = ratio;
    sm->cnt = 0u;
  }
}

// Y += X (the solved correction), row by row.
template <int K>
__global__ void __launch_bounds__(kBlock) eig_addx_kernel(double* __restrict__ Y, const double* __restrict__ X, long n) {
  const long i = (long)blockIdx.x * kBlock + threadIdx.x;
  if (i < n * K) Y[i] += X[i];
}

// U = Y R^-1 (row by row).
template <int K>
__global__ void __launch_bounds__(kBlock) eig_transform_kernel(const double* __restrict__ Y, double* __restrict__ U,
                                                               long n, const EigSmall* __restrict__ sm) {
  __shared__ double ri[K * K];
  if (threadIdx.x < K * K) ri[threadIdx.x] = sm->rinv[threadIdx.x];
  __syncthreads();
  const long row = (long)blockIdx.x * kBlock + threadIdx.x;
  if (row >= n) return;
  double y[K];
#pragma unroll
  for (int c = 0; c < K; ++c) y[c] = Y[row * K + c];
#pragma unroll
  for (int c = 0; c < K; ++c) {
    double u = 0.0;
#pragma unroll
    for (int a = 0; a <= c; ++a) u = fma(y[a], ri[a * K + c], u);
    U[row * K + c] = u;
  }
}

// Column maxima of |U| (exact, order-free) and the Rayleigh quotients: u^T A u and u^T M u per
// column, summed in tile order; the completing CTA writes colmax and lambda.
template <int K>
__global__ void __launch_bounds__(kBlock) eig_stats_kernel(const MeshDev* __restrict__ mds, const double* __restrict__ U,
                                                           double t, double* __restrict__ part, EigSmall* sm) {
  __shared__ double sh[2 * K * kBlock];
  __shared__ double smax[K][kBlock / 32];
  const MeshDev& md = mds[0];
  const long n = md.n;
  const int ntile = (int)((n + kBlock - 1) / kBlock);
  const long row = (long)blockIdx.x * kBlock + threadIdx.x;
  double acc[2 * K];
  double mx[K];
#pragma unroll
  for (int c = 0; c < K; ++c) {
    acc[c] = 0.0;
    acc[K + c] = 0.0;
    mx[c] = 0.0;
  }
  if (row < n) {
    double au[K], u[K];
    row_product<K>(md, md.A, row, GatherAoS64<K>{U}, au);
    const double m = md.M[row];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      u[c] = U[row * K + c];
      acc[c] = u[c] * au[c];
      acc[K + c] = m * u[c] * u[c];
      mx[c] = fabs(u[c]);
    }
  }
  // CTA maximum per column (warp shuffles, then the warps in order; max is exact)
#pragma unroll
  for (int c = 0; c < K; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx[c] = fmax(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
    if ((threadIdx.x & 31) == 0) smax[c][threadIdx.x >> 5] = mx[c];
  }
  block_sum<2 * K>(acc, sh);  // its barriers also publish smax
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < K; ++c) {
      double m = smax[c][0];
      for (int w = 1; w < kBlock / 32; ++w) m = fmax(m, smax[c][w]);
      part[(long)blockIdx.x * kEigStride + 2 * K + c] = m;
    }
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) part[(long)blockIdx.x * kEigStride + i] = acc[i];
  }
  if (!eig_publish(sm, ntile)) return;
  double tot[2 * K];
  eig_gather_sum<2 * K>(part, ntile, tot, sh);
  double cm[K];
  eig_gather_ext<K, false>(part, ntile, 2 * K, cm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < K; ++c) {
      sm->colmax[c] = cm[c];
      sm->lambda[c] = (tot[c] - tot[K + c]) / t;
    }
    sm->cnt = 0u;
  }
}

// The first row (in vertex order) of each column whose magnitude is within the band below the
// column maximum; its sign is the column's canonical sign.
template <int K>
__global__ void __launch_bounds__(kBlock) eig_sign_kernel(const double* __restrict__ U, long n,
                                                          double* __restrict__ part, EigSmall* sm) {
  __shared__ int smin[K][kBlock / 32];
  const int ntile = (int)((n + kBlock - 1) / kBlock);
  const long row = (long)blockIdx.x * kBlock + threadIdx.x;
  int first[K];
#pragma unroll
  for (int c = 0; c < K; ++c) {
    first[c] = INT_MAX;
    if (row < n) {
      const double thr = (1.0 - kSignBand) * __ldcg(&sm->colmax[c]);
      if (fabs(U[row * K + c]) >= thr) first[c] = (int)row;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) first[c] = min(first[c], __shfl_xor_sync(0xffffffffu, first[c], o));
    if ((threadIdx.x & 31) == 0) smin[c][threadIdx.x >> 5] = first[c];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < K; ++c) {
      int m = smin[c][0];
      for (int w = 1; w < kBlock / 32; ++w) m = min(m, smin[c][w]);
      part[(long)blockIdx.x * kEigStride + c] = (double)m;
    }
  }
  if (!eig_publish(sm, ntile)) return;
  double fr[K];
  eig_gather_ext<K, true>(part, ntile, 0, fr);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const long r = fr[c] < (double)n ? (long)fr[c] : 0;
      sm->sign_row[c] = (int)r;
      sm->sign[c] = U[r * K + c] < 0.0 ? -1.0 : 1.0;
    }
    sm->cnt = 0u;
  }
}

template <int K>
__global__ void __launch_bounds__(kBlock) eig_flip_kernel(double* __restrict__ U, long n, const EigSmall* __restrict__ sm) {
  const long row = (long)blockIdx.x * kBlock + threadIdx.x;
  if (row >= n) return;
#pragma unroll
  for (int c = 0; c < K; ++c) U[row * K + c] *= sm->sign[c];
}

// ---------------------------------------------------------------------------------------------
// Gradient through the fixed point.

// s_c = sign(sum_i M_i (Y R^-1)_ic U_ic): the canonical signs that turn Qraw = Y R^-1 into U*.
template <int K>
__global__ void __launch_bounds__(kBlock) eig_align_kernel(const double* __restrict__ Y, const double* __restrict__ U,
                                                           const double* __restrict__ M, long n,
                                                           double* __restrict__ part, EigSmall* sm) {
  __shared__ double sh[K * kBlock];
  __shared__ double ri[K * K];
  if (threadIdx.x < K * K) ri[threadIdx.x] = sm->rinv[threadIdx.x];
  __syncthreads();
  const int ntile = (int)((n + kBlock - 1) / kBlock);
  const long row = (long)blockIdx.x * kBlock + threadIdx.x;
  double acc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = 0.0;
  if (row < n) {
    double y[K];
#pragma unroll
    for (int c = 0; c < K; ++c) y[c] = Y[row * K + c];
    const double m = M[row];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      double q = 0.0;
#pragma unroll
      for (int a = 0; a <= c; ++a) q = fma(y[a], ri[a * K + c], q);
      acc[c] = m * q * U[row * K + c];
    }
  }
  block_sum<K>(acc, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < K; ++c) part[(long)blockIdx.x * kEigStride + c] = acc[c];
  if (!eig_publish(sm, ntile)) return;
  double tot[K];
  eig_gather_sum<K>(part, ntile, tot, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < K; ++c) sm->sign[c] = tot[c] < 0.0 ? -1.0 : 1.0;
    sm->cnt = 0u;
  }
}

// C0 = Qraw^T Qb (Qb = w diag(s)), then P = R^-1 Phi(C0) R^-T on the completing CTA.
template <int K>
__global__ void __launch_bounds__(kBlock) eig_qtq_kernel(const double* __restrict__ Y, const double* __restrict__ W,
                                                         long n, double* __restrict__ part, EigSmall* sm) {
  __shared__ double sh[K * K * kBlock];
  __shared__ double ri[K * K];
  __shared__ double sg[K];
  if (threadIdx.x < K * K) ri[threadIdx.x] = sm->rinv[threadIdx.x];
  if (threadIdx.x < K) sg[threadIdx.x] = sm->sign[threadIdx.x];
  __syncthreads();
  const int ntile = (int)((n + kBlock - 1) / kBlock);
  const long row = (long)blockIdx.x * kBlock + threadIdx.x;
  double acc[K * K];
#pragma unroll
  for (int i = 0; i < K * K; ++i) acc[i] = 0.0;
  if (row < n) {
    double y[K], q[K], b[K];
#pragma unroll
    for (int c = 0; c < K; ++c) y[c] = Y[row * K + c];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      double v = 0.0;
#pragma unroll
      for (int a = 0; a <= c; ++a) v = fma(y[a], ri[a * K + c], v);
      q[c] = v;
      b[c] = W[row * K + c] * sg[c];
    }
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
      for (int c = 0; c < K; ++c) acc[a * K + c] = q[a] * b[c];
  }
  block_sum<K * K>(acc, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < K * K; ++i) part[(long)blockIdx.x * kEigStride + i] = acc[i];
  if (!eig_publish(sm, ntile)) return;
  double c0[K * K];
  eig_gather_sum<K * K>(part, ntile, c0, sh);
  if (threadIdx.x != 0) return;
  double C[K][K], T[K][K];
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int c = 0; c < K; ++c) C[a][c] = a < c ? c0[a * K + c] : (a == c ? 0.5 * c0[a * K + c] : 0.0);
  // T = R^-1 C, then P = T R^-T
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int c = 0; c < K; ++c) {
      double v = 0.0;
#pragma unroll
      for (int e = 0; e < K; ++e) v = fma(ri[a * K + e], C[e][c], v);
      T[a][c] = v;
    }
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int c = 0; c < K; ++c) {
      double v = 0.0;
#pragma unroll
      for (int e = 0; e < K; ++e) v = fma(T[a][e], ri[c * K + e], v);
      sm->p[a * K + c] = v;
    }
  sm->cnt = 0u;
}

// Ybar = Qb R^-T - M Y (P + P^T), row by row.
template <int K>
__global__ void __launch_bounds__(kBlock) eig_ybar_kernel(const double* __restrict__ Y, const double* __restrict__ W,
                                                          const double* __restrict__ M, long n,
                                                          double* __restrict__ Yb, const EigSmall* __restrict__ sm) {
  __shared__ double ri[K * K];
  __shared__ double ps[K * K];  // P + P^T
  __shared__ double sg[K];
  if (threadIdx.x < K * K) {
    const int a = threadIdx.x / K, c = threadIdx.x % K;
    ri[threadIdx.x] = sm->rinv[threadIdx.x];
    ps[threadIdx.x] = sm->p[a * K + c] + sm->p[c * K + a];
  }
  if (threadIdx.x < K) sg[threadIdx.x] = sm->sign[threadIdx.x];
  __syncthreads();
  const long row = (long)blockIdx.x * kBlock + threadIdx.x;
  if (row >= n) return;
  double y[K], b[K];
#pragma unroll
  for (int c = 0; c < K; ++c) {
    y[c] = Y[row * K + c];
    b[c] = W[row * K + c] * sg[c];
  }
  const double m = M[row];
#pragma unroll
  for (int c = 0; c < K; ++c) {
    double v = 0.0, u = 0.0;
#pragma unroll
    for (int a = c; a < K; ++a) v = fma(b[a], ri[c * K + a], v);  // (Qb R^-T)_c = sum_a Qb_a Rinv[c][a]
#pragma unroll
    for (int a = 0; a < K; ++a) u = fma(y[a], ps[a * K + c], u);
    Yb[row * K + c] = fma(-m, u, v);
  }
}

// W = gU + M X (the next Neumann term).
template <int K>
__global__ void __launch_bounds__(kBlock) eig_wnext_kernel(const double* __restrict__ gU, const double* __restrict__ X,
                                                           const double* __restrict__ M, long n, double* __restrict__ W) {
  const long row = (long)blockIdx.x * kBlock + threadIdx.x;
  if (row >= n) return;
  const double m = M[row];
#pragma unroll
  for (int c = 0; c < K; ++c) W[row * K + c] = fma(m, X[row * K + c], gU[row * K + c]);
}

// Mass weights of the Gram matrix's term: w_i = -Y_i P Y_i^T.
template <int K>
__global__ void __launch_bounds__(kBlock) eig_massw_kernel(const double* __restrict__ Y, long n,
                                                           double* __restrict__ wm, const EigSmall* __restrict__ sm) {
  __shared__ double ps[K * K];
  if (threadIdx.x < K * K) ps[threadIdx.x] = sm->p[threadIdx.x];
  __syncthreads();
  const long row = (long)blockIdx.x * kBlock + threadIdx.x;
  if (row >= n) return;
  double y[K];
#pragma unroll
  for (int c = 0; c < K; ++c) y[c] = Y[row * K + c];
  double v = 0.0;
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int c = 0; c < K; ++c) v = fma(y[a] * ps[a * K + c], y[c], v);
  wm[row] = -v;
}

}  // namespace

// Workspace layout (doubles): Y, Ybar, X, W [n][4] each; mass weights [n]; tile partials
// [ntile][kEigStride]; EigSmall.
struct EigLayout {
  double *Y, *Yb, *X, *W, *wm, *part;
  EigSmall* sm;
  EigLayout(double* ws, long n) {
    const long ntile = (n + kBlock - 1) / kBlock;
    Y = ws;
    Yb = Y + kMaxK * n;
    X = Yb + kMaxK * n;
    W = X + kMaxK * n;
    wm = W + kMaxK * n;
    part = wm + n;
    sm = reinterpret_cast<EigSmall*>(part + kEigStride * ntile);
  }
};

size_t eig_workspace_doubles(long n) {
  const long ntile = (n + kBlock - 1) / kBlock;
  return (size_t)(4 * kMaxK * n + n + kEigStride * ntile) + (sizeof(EigSmall) + 7) / 8 + 1;
}

cudaError_t eig_reset(double* ws, long n, cudaStream_t st) {
  return cudaMemsetAsync(EigLayout(ws, n).sm, 0, sizeof(EigSmall), st);
}

template <int K>
static cudaError_t eig_step_k(double* ws, const double* M, long n, double* U, cudaStream_t st) {
  const long ntile = (n + kBlock - 1) / kBlock;
  const EigLayout L(ws, n);
  double* Y = L.Y;
  double* part = L.part;
  EigSmall* sm = L.sm;
  {
    IG_PROF("eig_gram", st);
    eig_gram_kernel<K><<<(unsigned)ntile, kBlock, 0, st>>>(Y, M, n, part, sm);
  }
  {
    IG_PROF("eig_transform", st);
    eig_transform_kernel<K><<<(unsigned)ntile, kBlock, 0, st>>>(Y, U, n, sm);
  }
  return cudaGetLastError();
}

cudaError_t eig_step(int k, double* ws, const double* M, long n, double* U, cudaStream_t st) {
  switch (k) {
    case 1: return eig_step_k<1>(ws, M, n, U, st);
    case 2: return eig_step_k<2>(ws, M, n, U, st);
    case 3: return eig_step_k<3>(ws, M, n, U, st);
    case 4: return eig_step_k<4>(ws, M, n, U, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int K>
static cudaError_t eig_finish_k(const MeshDev* mds, double t, double* ws, long n, double* U, cudaStream_t st) {
  const long ntile = (n + kBlock - 1) / kBlock;
  const EigLayout L(ws, n);
  double* part = L.part;
  EigSmall* sm = L.sm;
  {
    IG_PROF("eig_stats", st);
    eig_stats_kernel<K><<<(unsigned)ntile, kBlock, 0, st>>>(mds, U, t, part, sm);
  }
  {
    IG_PROF("eig_sign", st);
    eig_sign_kernel<K><<<(unsigned)ntile, kBlock, 0, st>>>(U, n, part, sm);
  }
  {
    IG_PROF("eig_flip", st);
    eig_flip_kernel<K><<<(unsigned)ntile, kBlock, 0, st>>>(U, n, sm);
  }
  return cudaGetLastError();
}

cudaError_t eig_finish(int k, const MeshDev* mds, double t, double* ws, long n, double* U, cudaStream_t st) {
  switch (k) {
    case 1: return eig_finish_k<1>(mds, t, ws, n, U, st);
    case 2: return eig_finish_k<2>(mds, t, ws, n, U, st);
    case 3: return eig_finish_k<3>(mds, t, ws, n, U, st);
    case 4: return eig_finish_k<4>(mds, t, ws, n, U, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t eig_read(double* ws, long n, int k, double* lambda_host, int* fail_host, cudaStream_t st) {
  EigSmall* sm = EigLayout(ws, n).sm;
  cudaError_t e = cudaSuccess;
  if (lambda_host) e = cudaMemcpyAsync(lambda_host, sm->lambda, sizeof(double) * k, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && fail_host) e = cudaMemcpyAsync(fail_host, &sm->fail, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

// Gradient step helpers (see the header comment). Y: the workspace's Y = (M + tL)^-1 M U*.
template <int K>
static cudaError_t eig_vjp_prepare_k(double* ws, const double* M, long n, const double* U, const double* gU,
                                     cudaStream_t st) {
  const long ntile = (n + kBlock - 1) / kBlock;
  const EigLayout L(ws, n);
  {
    IG_PROF("eig_gram", st);
    eig_gram_kernel<K><<<(unsigned)ntile, kBlock, 0, st>>>(L.Y, M, n, L.part, L.sm);
  }
  {
    IG_PROF("eig_align", st);
    eig_align_kernel<K><<<(unsigned)ntile, kBlock, 0, st>>>(L.Y, U, M, n, L.part, L.sm);
  }
  cudaError_t e = cudaMemcpyAsync(L.W, gU, sizeof(double) * K * n, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int K>
static cudaError_t eig_vjp_ybar_k(double* ws, const double* M, long n, cudaStream_t st) {
  const long ntile = (n + kBlock - 1) / kBlock;
  const EigLayout L(ws, n);
  {
    IG_PROF("eig_qtq", st);
    eig_qtq_kernel<K><<<(unsigned)ntile, kBlock, 0, st>>>(L.Y, L.W, n, L.part, L.sm);
  }
  {
    IG_PROF("eig_ybar", st);
    eig_ybar_kernel<K><<<(unsigned)ntile, kBlock, 0, st>>>(L.Y, L.W, M, n, L.Yb, L.sm);
  }
  return cudaGetLastError();
}

template <int K>
static cudaError_t eig_vjp_next_k(double* ws, const double* M, long n, const double* gU, cudaStream_t st) {
  const long ntile = (n + kBlock - 1) / kBlock;
  const EigLayout L(ws, n);
  IG_PROF("eig_wnext", st);
  eig_wnext_kernel<K><<<(unsigned)ntile, kBlock, 0, st>>>(gU, L.X, M, n, L.W);
  return cudaGetLastError();
}

template <int K>
static cudaError_t eig_vjp_massw_k(double* ws, long n, cudaStream_t st) {
  const long ntile = (n + kBlock - 1) / kBlock;
  const EigLayout L(ws, n);
  IG_PROF("eig_massw", st);
  eig_massw_kernel<K><<<(unsigned)ntile, kBlock, 0, st>>>(L.Y, n, L.wm, L.sm);
  return cudaGetLastError();
}

cudaError_t eig_vjp_prepare(int k, double* ws, const double* M, long n, const double* U, const double* gU,
                            cudaStream_t st) {
  switch (k) {
    case 1: return eig_vjp_prepare_k<1>(ws, M, n, U, gU, st);
    case 2: return eig_vjp_prepare_k<2>(ws, M, n, U, gU, st);
    case 3: return eig_vjp_prepare_k<3>(ws, M, n, U, gU, st);
    case 4: return eig_vjp_prepare_k<4>(ws, M, n, U, gU, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t eig_vjp_ybar(int k, double* ws, const double* M, long n, cudaStream_t st) {
  switch (k) {
    case 1: return eig_vjp_ybar_k<1>(ws, M, n, st);
    case 2: return eig_vjp_ybar_k<2>(ws, M, n, st);
    case 3: return eig_vjp_ybar_k<3>(ws, M, n, st);
    case 4: return eig_vjp_ybar_k<4>(ws, M, n, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t eig_vjp_next(int k, double* ws, const double* M, long n, const double* gU, cudaStream_t st) {
  switch (k) {
    case 1: return eig_vjp_next_k<1>(ws, M, n, gU, st);
    case 2: return eig_vjp_next_k<2>(ws, M, n, gU, st);
    case 3: return eig_vjp_next_k<3>(ws, M, n, gU, st);
    case 4: return eig_vjp_next_k<4>(ws, M, n, gU, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t eig_vjp_massw(int k, double* ws, long n, cudaStream_t st) {
  switch (k) {
    case 1: return eig_vjp_massw_k<1>(ws, n, st);
    case 2: return eig_vjp_massw_k<2>(ws, n, st);
    case 3: return eig_vjp_massw_k<3>(ws, n, st);
    case 4: return eig_vjp_massw_k<4>(ws, n, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int K>
static cudaError_t eig_warm_k(const MeshDev* mds, double* ws, long n, const double* U, cudaStream_t st) {
  const long ntile = (n + kBlock - 1) / kBlock;
  const EigLayout L(ws, n);
  IG_PROF("eig_warm", st);
  eig_warm_kernel<K><<<(unsigned)ntile, kBlock, 0, st>>>(mds, U, L.Y, L.Yb, L.part, L.sm);
  return cudaGetLastError();
}

cudaError_t eig_warm(int k, const MeshDev* mds, double* ws, long n, const double* U, double* tol_ratio_host,
                     cudaStream_t st) {
  cudaError_t e;
  switch (k) {
    case 1: e = eig_warm_k<1>(mds, ws, n, U, st); break;
    case 2: e = eig_warm_k<2>(mds, ws, n, U, st); break;
    case 3: e = eig_warm_k<3>(mds, ws, n, U, st); break;
    case 4: e = eig_warm_k<4>(mds, ws, n, U, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(tol_ratio_host, &EigLayout(ws, n).sm->tol_ratio, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

cudaError_t eig_addx(int k, double* ws, long n, cudaStream_t st) {
  const EigLayout L(ws, n);
  const long count = (long)k * n;
  IG_PROF("eig_addx", st);
  switch (k) {
    case 1: eig_addx_kernel<1><<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(L.Y, L.X, n); break;
    case 2: eig_addx_kernel<2><<<(unsigned)((count + kBlock - 1) / kBlock), kBlock, 0, st>>>(L.Y, L.X, n); break;
    case 3: eig_addx_kernel<3><<<(unsigned)((count + kBlock - 1) / kBlock), kBlock, 0, st>>>(L.Y, L.X, n); break;
    case 4: eig_addx_kernel<4><<<(unsigned)((count + kBlock - 1) / kBlock), kBlock, 0, st>>>(L.Y, L.X, n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

EigBuffers eig_buffers(double* ws, long n) {
  const EigLayout L(ws, n);
  return EigBuffers{L.Y, L.Yb, L.X, L.W, L.wm};
}

}  // namespace ig
