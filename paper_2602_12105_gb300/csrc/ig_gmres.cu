// ig_gmres.cu -- restarted GMRES (Saad and Schultz's generalized minimal residual method) on device
// vectors, the linear solver of the framework's implicit layers (the adjoint equations of a fixed
// point, with the Jacobian given only as a product). Used by the fixed-point adjoint of the
// geodesic ADMM, where N = 6 m unknowns and one product costs one constrained Laplacian solve.
//
// One Arnoldi step k (basis v_0 .. v_k, t = A v_k):
//   classical Gram-Schmidt applied twice (h = V^T t, t -= V h, twice; the second pass restores the
//   orthogonality the first loses in floating point), h_{k+1} = |t|, v_{k+1} = t / h_{k+1};
//   the Hessenberg column is rotated by the earlier Givens rotations, a new rotation zeroes
//   h_{k+1}, and |g_{k+1}| (g the rotated |r_0| e_1) is the residual norm of the least-squares
//   iterate, read by the host to decide whether to stop.
// At the end of a cycle the triangular system R c = g is solved and x += V c; a restart forms the
// true residual rhs - A x and starts again from it.
//
// Every inner product is deterministic: per-CTA partial sums over fixed chunks (each thread keeps
// its chunk of t in registers while the CTA walks the basis vectors), then one CTA per product
// adds the partials in CTA order. The small Hessenberg arithmetic runs on one device thread.
#include <cmath>

#include "ig_internal.cuh"

namespace ig {

namespace {

constexpr int kGmPer = 4;                       // elements of t per thread in the dot kernel
constexpr long kGmChunk = (long)kBlock * kGmPer;  // elements per CTA
constexpr int kGmMaxRestart = 100;

// Sum over the CTA in a fixed order; the result is valid in thread 0. sh: kBlock / 32 doubles.
__device__ double gm_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = threadIdx.x < kBlock / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

// part[j][cta] = sum over the CTA's chunk of Vb_j . t, for j < nvec (Vb_j = Vb + j ldv).
__global__ void __launch_bounds__(kBlock) gm_dots_kernel(const double* __restrict__ Vb, long ldv, int nvec,
                                                         const double* __restrict__ t, long N,
                                                         double* __restrict__ part) {
  __shared__ double sh[kBlock / 32];
  const long base = (long)blockIdx.x * kGmChunk + threadIdx.x;
  double tv[kGmPer];
#pragma unroll
  for (int s = 0; s < kGmPer; ++s) {
    const long i = base + (long)s * kBlock;
    tv[s] = i < N ? t[i] : 0.0;
  }
  for (int j = 0; j < nvec; ++j) {
    const double* vj = Vb + (long)j * ldv;
    double acc = 0.0;
#pragma unroll
    for (int s = 0; s < kGmPer; ++s) {
      const long i = base + (long)s * kBlock;
      if (i < N) acc = fma(vj[i], tv[s], acc);
    }
    acc = gm_block_sum(acc, sh);
    if (threadIdx.x == 0) part[(long)j * gridDim.x + blockIdx.x] = acc;
  }
}

// out[j] = sum over CTAs of part[j][cta], one CTA per j, in a fixed order.
__global__ void __launch_bounds__(kBlock) gm_reduce_kernel(const double* __restrict__ part, int nparts,
                                                           double* __restrict__ out) {
  __shared__ double sh[kBlock / 32];
  const double* pj = part + (long)blockIdx.x * nparts;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += kBlock) acc += pj[i];
  acc = gm_block_sum(acc, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

// t += sign * sum_j coef_j Vb_j.
__global__ void __launch_bounds__(kBlock) gm_axpy_kernel(double* __restrict__ t, const double* __restrict__ Vb,
                                                         long ldv, int nvec, const double* __restrict__ coef,
                                                         double sign, long N) {
  for (long i = (long)blockIdx.x * kBlock + threadIdx.x; i < N; i += (long)gridDim.x * kBlock) {
    double acc = 0.0;
    for (int j = 0; j < nvec; ++j) acc = fma(coef[j], Vb[(long)j * ldv + i], acc);
    t[i] = fma(sign, acc, t[i]);
  }
}

// dst = a * scal[0] (b null), or dst = a - b.
// dst may be a (an in-place scale), so neither is marked __restrict__.
__global__ void __launch_bounds__(kBlock) gm_vec_kernel(double* dst, const double* a, const double* __restrict__ b,
                                                        const double* __restrict__ scal, long N) {
  for (long i = (long)blockIdx.x * kBlock + threadIdx.x; i < N; i += (long)gridDim.x * kBlock)
    dst[i] = b ? a[i] - b[i] : a[i] * scal[0];
}

// The small state of a cycle, in one device array of gm_small_size(R) doubles.
struct Small {
  double* H;      // (R + 1) x R Hessenberg, column-major, rotated into upper triangular
  double* cs;     // [R] Givens cosines
  double* sn;     // [R] Givens sines
  double* g;      // [R + 1] rotated |r_0| e_1
  double* h1;     // [R + 1] first Gram-Schmidt pass
  double* h2;     // [R + 1] second pass
  double* nn;     // [1] |t|^2
  double* inv;    // [1] 1 / |t| (0 when |t| = 0)
  double* resid;  // [1] |g_{k+1}|
  double* coef;   // [R + 1] the cycle's least-squares coefficients
};

__host__ __device__ inline long gm_small_size(int R) { return (long)(R + 1) * R + 2L * R + 4L * (R + 1) + 3; }

__host__ __device__ inline Small gm_small(double* p, int R) {
  Small s;
  s.H = p;
  s.cs = s.H + (long)(R + 1) * R;
  s.sn = s.cs + R;
  s.g = s.sn + R;
  s.h1 = s.g + R + 1;
  s.h2 = s.h1 + R + 1;
  s.nn = s.h2 + R + 1;
  s.inv = s.nn + 1;
  s.resid = s.inv + 1;
  s.coef = s.resid + 1;
  return s;
}

// Start of a cycle from |r|^2 in nn: g = |r| e_1, inv = 1 / |r|, resid = |r|.
__global__ void gm_start_kernel(double* small, int R) {
  const Small s = gm_small(small, R);
  const double hn = sqrt(fmax(s.nn[0], 0.0));
  for (int i = 0; i <= R; ++i) s.g[i] = 0.0;
  s.g[0] = hn;
  s.inv[0] = hn > 0.0 ? 1.0 / hn : 0.0;
  s.resid[0] = hn;
}

// Arnoldi column k: h = h1 + h2, h_{k+1} = |t|; earlier rotations, a new one, the residual estimate.
__global__ void gm_arnoldi_kernel(double* small, int R, int k) {
  const Small s = gm_small(small, R);
  double* col = s.H + (long)k * (R + 1);
  for (int j = 0; j <= k; ++j) col[j] = s.h1[j] + s.h2[j];
  const double hn = sqrt(fmax(s.nn[0], 0.0));
  col[k + 1] = hn;
  for (int i = 0; i < k; ++i) {
    const double a = col[i], b = col[i + 1];
    col[i] = s.cs[i] * a + s.sn[i] * b;
    col[i + 1] = -s.sn[i] * a + s.cs[i] * b;
  }
  const double r = hypot(col[k], col[k + 1]);
  const double c = r > 0.0 ? col[k] / r : 1.0;
  const double sn = r > 0.0 ? col[k + 1] / r : 0.0;
  col[k] = r;
  col[k + 1] = 0.0;
  s.cs[k] = c;
  s.sn[k] = sn;
  s.g[k + 1] = -sn * s.g[k];
  s.g[k] = c * s.g[k];
  s.inv[0] = hn > 0.0 ? 1.0 / hn : 0.0;
  s.resid[0] = fabs(s.g[k + 1]);
}

// coef = R^-1 g over the cycle's kk columns (R the rotated Hessenberg); a zero pivot gives 0.
__global__ void gm_backsolve_kernel(double* small, int R, int kk) {
  const Small s = gm_small(small, R);
  for (int i = kk - 1; i >= 0; --i) {
    double v = s.g[i];
    for (int j = i + 1; j < kk; ++j) v -= s.H[i + (long)j * (R + 1)] * s.coef[j];
    const double d = s.H[i + (long)i * (R + 1)];
    s.coef[i] = d != 0.0 ? v / d : 0.0;
  }
}

struct DevBuf {
  double* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

int vec_grid(long N) {
  const long b = (N + kBlock - 1) / kBlock;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t gmres_solve(const std::function<cudaError_t(const double*, double*)>& apply, const double* rhs, double* x,
                        long N, int restart, int max_iter, double rel_tol, cudaStream_t st, GmresResult* res) {
  res->iterations = 0;
  res->rel_resid = 0.0;
  res->converged = 0;
  if (N <= 0 || restart < 1 || restart > kGmMaxRestart || max_iter < 1) return cudaErrorInvalidValue;
  const int R = restart;
  const int G = (int)((N + kGmChunk - 1) / kGmChunk);
  const long nsmall = gm_small_size(R);
  DevBuf buf;
  const size_t count = (size_t)(R + 1) * N + (size_t)(R + 1) * G + (size_t)nsmall;
  cudaError_t e = cudaMalloc(&buf.p, sizeof(double) * count);
  if (e != cudaSuccess) return e;
  double* basis = buf.p;
  double* part = basis + (size_t)(R + 1) * N;
  double* small = part + (size_t)(R + 1) * G;
  const Small s = gm_small(small, R);
  const int vg = vec_grid(N);

  auto dots = [&](const double* Vb, int nvec, const double* t, double* out) -> cudaError_t {
    {
      IG_PROF("gmres_dots", st);
      gm_dots_kernel<<<G, kBlock, 0, st>>>(Vb, N, nvec, t, N, part);
    }
    cudaError_t e2 = cudaGetLastError();
    if (e2 != cudaSuccess) return e2;
    gm_reduce_kernel<<<nvec, kBlock, 0, st>>>(part, G, out);
    return cudaGetLastError();
  };
  auto axpy = [&](double* t, const double* Vb, int nvec, const double* coef, double sign) -> cudaError_t {
    IG_PROF("gmres_axpy", st);
    gm_axpy_kernel<<<vg, kBlock, 0, st>>>(t, Vb, N, nvec, coef, sign, N);
    return cudaGetLastError();
  };
  auto read_resid = [&](double* out) -> cudaError_t {
    cudaError_t e2 = cudaMemcpyAsync(out, s.resid, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
    return e2;
  };

  if ((e = cudaMemsetAsync(x, 0, sizeof(double) * N, st)) != cudaSuccess) return e;
  // |rhs|, and the first cycle starts from r = rhs (x = 0)
  if ((e = dots(rhs, 1, rhs, s.nn)) != cudaSuccess) return e;
  gm_start_kernel<<<1, 1, 0, st>>>(small, R);
  double bnorm = 0.0;
  if ((e = cudaGetLastError()) != cudaSuccess || (e = read_resid(&bnorm)) != cudaSuccess) return e;
  if (!std::isfinite(bnorm)) {
    res->rel_resid = bnorm;
    return cudaSuccess;
  }
  if (bnorm == 0.0) {
    res->converged = 1;
    return cudaSuccess;
  }
  gm_vec_kernel<<<vg, kBlock, 0, st>>>(basis, rhs, nullptr, s.inv, N);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int iters = 0;
  double rel = 1.0;
  bool done = false, bad = false;
  while (!done) {
    int kk = 0;
    for (int k = 0; k < R && iters < max_iter; ++k) {
      double* t = basis + (size_t)(k + 1) * N;
      if ((e = apply(basis + (size_t)k * N, t)) != cudaSuccess) return e;
      if ((e = dots(basis, k + 1, t, s.h1)) != cudaSuccess) return e;
      if ((e = axpy(t, basis, k + 1, s.h1, -1.0)) != cudaSuccess) return e;
      if ((e = dots(basis, k + 1, t, s.h2)) != cudaSuccess) return e;
      if ((e = axpy(t, basis, k + 1, s.h2, -1.0)) != cudaSuccess) return e;
      if ((e = dots(t, 1, t, s.nn)) != cudaSuccess) return e;
      gm_arnoldi_kernel<<<1, 1, 0, st>>>(small, R, k);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      gm_vec_kernel<<<vg, kBlock, 0, st>>>(t, t, nullptr, s.inv, N);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      ++iters;
      kk = k + 1;
      double r = 0.0;
      if ((e = read_resid(&r)) != cudaSuccess) return e;
      rel = r / bnorm;
      if (!std::isfinite(rel)) {
        bad = true;
        break;
      }
      if (rel <= rel_tol) {
        done = true;
        break;
      }
    }
    if (kk > 0 && !bad) {
      gm_backsolve_kernel<<<1, 1, 0, st>>>(small, R, kk);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = axpy(x, basis, kk, s.coef, 1.0)) != cudaSuccess) return e;
    }
    if (done || bad || iters >= max_iter) break;
    // restart from the true residual rhs - A x
    if ((e = apply(x, basis + N)) != cudaSuccess) return e;
    gm_vec_kernel<<<vg, kBlock, 0, st>>>(basis, rhs, basis + N, nullptr, N);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = dots(basis, 1, basis, s.nn)) != cudaSuccess) return e;
    gm_start_kernel<<<1, 1, 0, st>>>(small, R);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    double r = 0.0;
    if ((e = read_resid(&r)) != cudaSuccess) return e;
    rel = r / bnorm;
    if (!std::isfinite(rel)) break;
    if (rel <= rel_tol) {
      done = true;
      break;
    }
    gm_vec_kernel<<<vg, kBlock, 0, st>>>(basis, basis, nullptr, s.inv, N);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // the basis is freed on return: finish its last users first
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  res->iterations = iters;
  res->rel_resid = rel;
  res->converged = done ? 1 : 0;
  return cudaSuccess;
}

}  // namespace ig
