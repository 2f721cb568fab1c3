// ig_vjp.cu -- vector-Jacobian product of the smoothing step with respect to the positions.
//
// The adjoint rule for linear solves (§5.2; Eq. 3 of §3.1 with f = A(V) U - M(V) B) gives, with
// Lambda = A^-1 dl/dU,
//   dl/dV = <Lambda, d(M B)/dV - (dA/dV) U>,   dl/dB = M Lambda,   dl/dt = -<Lambda, L U>.
// With A = M + t L, per face f this is the gradient of the scalar
//   E_f = w_a * area_f + sum_c omega_c * cot_c,
//   w_a     = (1/3) sum_{v in f} <Lambda_v, B_v - U_v>,
//   omega_c = -(t/2) <Lambda_a - Lambda_b, U_a - U_b>   ((a, b) the edge opposite corner c),
// with the coefficients held fixed. Writing d_c for the edge opposite corner c (d_0 = p2 - p1,
// d_1 = p0 - p2, d_2 = p1 - p0), N = d_1 x d_2, s = |N|, dot_c = d_{c+1}.d_{c+2} (so
// cot_c = -dot_c / s) and P = -sum_c omega_c dot_c, E_f = P / s + w_a s / 2 and
//   grad_{p_c} E_f = [ -omega_c (d_{c+2} - d_{c+1}) + (omega_{c+1} - omega_{c+2}) d_c ] / s
//                    + (w_a / 2 - P / s^2) (N x d_c) / s.
// (The CPU oracle reaches the same numbers through the per-corner cotangent gradients.)
//
// A loss may also depend on V through the mass directly (the M-norm loss of the inverse-fairing
// problem, §7.1): with per-vertex weights w, d(sum_i M_i w_i)/dV adds w_v / 3 per vertex of the
// face to w_a (M_i = sum over the faces at i of area / 3); the kernel's MODE selects the solve
// terms alone (0), both (1) or the mass term alone (2, no U, B or Lambda read).
//
// K6a (face-parallel) writes the three per-corner gradients of each face to gface [m][9] and a
// per-tile partial of dl/dt; K6b (vertex-parallel) gathers gface over the vertex's incidence
// list in face order (atomic-free, deterministic) and adds M Lambda where B is V.
#include "ig_internal.cuh"

namespace ig {

namespace {

constexpr int kFaceTile = 256;

// MODE 0: the solve terms; 1: the solve terms and the mass weights; 2: the mass weights alone.
template <int K, int MODE>
__global__ void __launch_bounds__(256) vjp_face_kernel(const MeshDev* __restrict__ mds,
                                                       const CallDev* __restrict__ calls,
                                                       const int2* __restrict__ ftiles) {
  __shared__ double sh[8];
  __shared__ int s_last;
  const int2 tl = ftiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const CallDev& cl = calls[tl.x];
  const double* __restrict__ V = cl.V;
  const double* __restrict__ Bsrc = cl.b_is_V ? cl.V : cl.B;
  const int bstride = cl.bstride;
  const double* __restrict__ U = cl.U;
  double* __restrict__ gt = cl.gt;
  const double tval = cl.t;
  const int ntl = (md.m + kFaceTile - 1) / kFaceTile;
  const int f = tl.y * kFaceTile + threadIdx.x;
  const double* __restrict__ lam = md.lam;
  double gt_part = 0.0;
  if (f < md.m) {
    int vid[3];
    double P[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      vid[c] = __ldg(md.F + 3 * f + c);
#pragma unroll
      for (int d = 0; d < 3; ++d) P[c][d] = __ldg(V + 3 * (long)vid[c] + d);
    }
    double dd[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      dd[0][d] = P[2][d] - P[1][d];
      dd[1][d] = P[0][d] - P[2][d];
      dd[2][d] = P[1][d] - P[0][d];
    }
    double N[3];
    N[0] = dd[1][1] * dd[2][2] - dd[1][2] * dd[2][1];
    N[1] = dd[1][2] * dd[2][0] - dd[1][0] * dd[2][2];
    N[2] = dd[1][0] * dd[2][1] - dd[1][1] * dd[2][0];
    const double s2 = N[0] * N[0] + N[1] * N[1] + N[2] * N[2];
    const double inv_s = rsqrt(s2);
    double dot[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int a = (c + 1) % 3, b = (c + 2) % 3;
      dot[c] = dd[a][0] * dd[b][0] + dd[a][1] * dd[b][1] + dd[a][2] * dd[b][2];
    }
    // per-vertex <Lambda_v, B_v - U_v> and the per-corner <dLambda, dU>; with mass weights w,
    // d(sum_i M_i w_i)/dV adds sum_f ((1/3) sum_{v in f} w_v) grad area_f, i.e. w_v to the sum
    double wa = 0.0;
    double omega[3] = {0.0, 0.0, 0.0};
    if constexpr (MODE != 2) {
      double L[3][K], Uv[3][K];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          L[c][k] = lam[(long)vid[c] * K + k];
          Uv[c][k] = U[(long)vid[c] * K + k];
          wa = fma(L[c][k], Bsrc[(long)vid[c] * bstride + k] - Uv[c][k], wa);
        }
      }
      const double mt2 = -0.5 * tval;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        double lu = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) lu = fma(L[a][k] - L[b][k], Uv[a][k] - Uv[b][k], lu);
        omega[c] = mt2 * lu;
        // dl/dt = -<Lambda, L U> = -sum_c (cot_c / 2) lu_c = sum_c (dot_c / s / 2) lu_c
        if (gt) gt_part = fma(0.5 * dot[c] * inv_s, lu, gt_part);
      }
    }
    if constexpr (MODE != 0) wa += (__ldg(cl.wm + vid[0]) + __ldg(cl.wm + vid[1])) + __ldg(cl.wm + vid[2]);
    wa *= (1.0 / 3.0);
    const double Pv = -(omega[0] * dot[0] + omega[1] * dot[1] + omega[2] * dot[2]);
    const double coef = (0.5 * wa - Pv * inv_s * inv_s) * inv_s;
    double g[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int a = (c + 1) % 3, b = (c + 2) % 3;
      const double om = omega[c] * inv_s;
      const double dom = (omega[a] - omega[b]) * inv_s;
      double nxd[3];
      nxd[0] = N[1] * dd[c][2] - N[2] * dd[c][1];
      nxd[1] = N[2] * dd[c][0] - N[0] * dd[c][2];
      nxd[2] = N[0] * dd[c][1] - N[1] * dd[c][0];
#pragma unroll
      for (int d = 0; d < 3; ++d)
        g[3 * c + d] = fma(coef, nxd[d], fma(dom, dd[c][d], -om * (dd[b][d] - dd[a][d])));
    }
    double* out = md.gface + 9 * (long)f;
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i] = g[i];
  }
  if (gt == nullptr) return;
  // deterministic reduction of dl/dt: warp shuffle, CTA partial, last CTA adds partials in order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gt_part += __shfl_xor_sync(0xffffffffu, gt_part, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = gt_part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < 8; ++w) tot += sh[w];
    md.part[tl.y] = tot;
    __threadfence();
    const unsigned prev = atomicAdd(&md.s->cnt[3], 1u);
    s_last = (prev == (unsigned)ntl - 1u);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double tot = 0.0;
  for (int b = threadIdx.x; b < ntl; b += blockDim.x) tot += __ldcg(md.part + b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    double all = 0.0;
    for (int w = 0; w < 8; ++w) all += sh[w];
    *gt = all;
    md.s->cnt[3] = 0u;
  }
}

template <int K>
__global__ void __launch_bounds__(256) vjp_gather_kernel(const MeshDev* __restrict__ mds,
                                                         const CallDev* __restrict__ calls,
                                                         const int2* __restrict__ rtiles) {
  const int2 tl = rtiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const int v = tl.y * 256 + threadIdx.x;
  if (v >= md.n) return;
  const int b_is_V = calls[tl.x].b_is_V;
  double* __restrict__ gV = calls[tl.x].gV;
  double* __restrict__ gB = calls[tl.x].gB;
  double g0 = 0.0, g1 = 0.0, g2 = 0.0;
  const int e0 = __ldg(md.incptr + v), e1 = __ldg(md.incptr + v + 1);
  for (int e = e0; e < e1; ++e) {
    const int fc = __ldg(&md.inc[e].x);
    const double* src = md.gface + 9 * (long)(fc >> 2) + 3 * (fc & 3);
    g0 += src[0];
    g1 += src[1];
    g2 += src[2];
  }
  const double mass = md.M[v];
  if (b_is_V) {
    g0 = fma(mass, md.lam[(long)v * K + 0], g0);
    g1 = fma(mass, md.lam[(long)v * K + 1], g1);
    g2 = fma(mass, md.lam[(long)v * K + 2], g2);
  }
  gV[3 * (long)v + 0] = g0;
  gV[3 * (long)v + 1] = g1;
  gV[3 * (long)v + 2] = g2;
  if (gB) {
#pragma unroll
    for (int k = 0; k < K; ++k) gB[(long)v * K + k] = mass * md.lam[(long)v * K + k];
  }
}

template <int K>
cudaError_t vjp_k(Group& g, int mode, cudaStream_t st) {
  {
    IG_PROF("vjp_face", st);
    if (mode == 0) vjp_face_kernel<K, 0><<<g.nface_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.face_tiles);
    else if (mode == 1) vjp_face_kernel<K, 1><<<g.nface_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.face_tiles);
    else vjp_face_kernel<K, 2><<<g.nface_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.face_tiles);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    IG_PROF("vjp_gather", st);
    vjp_gather_kernel<K><<<g.nrow_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.row_tiles);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_vjp(Group& g, int k, cudaStream_t st, int mode) {
  if (mode == 2) return vjp_k<1>(g, 2, st);
  switch (k) {
    case 1: return vjp_k<1>(g, mode, st);
    case 2: return vjp_k<2>(g, mode, st);
    case 3: return vjp_k<3>(g, mode, st);
    case 4: return vjp_k<4>(g, mode, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ig
