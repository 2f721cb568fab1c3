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
//
// FP32 face geometry (the mode whose operator was assembled from FP32 cotangents): a vertex pass
// splits U and Lambda into hi/lo floats and forms w_v = <Lambda_v, B_v - U_v> per vertex; K6a
// evaluates the same formula in FP32 with every difference of neighbouring values (edges, U_a -
// U_b, Lambda_a - Lambda_b) taken as (hi_a - hi_b) + (lo_a - lo_b), and slivers (sin theta < 1e-2
// at a corner, the test of the assembly) in FP64; gface is then [m][3][4] float (one 16-byte row
// per corner) and K6b adds in FP32. The FP64 solve terms of B = V (M Lambda) stay FP64.
#include "ig_f32.cuh"
#include "ig_internal.cuh"

namespace ig {

namespace {

constexpr int kFaceTile = 256;

// MODE 0: the solve terms; 1: the solve terms and the mass weights; 2: the mass weights alone.
// CLAMP: some mesh of the group clamps its cotangents (compiled out otherwise: this kernel is bound
// by FP64 instructions).
template <int K, int MODE, bool CLAMP>
__global__ void __launch_bounds__(256) vjp_face_kernel(const MeshDev* __restrict__ mds,
                                                       const CallDev* __restrict__ calls,
                                                       const int2* __restrict__ ftiles) {
  __shared__ double sh[8];
  __shared__ int s_last;
  const int2 tl = ftiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const CallDev& cl = calls[tl.x];
  const double* __restrict__ V = cl.V;
  const double* __restrict__ wvert = md.z;  // per-vertex weights (vjp_vertex_kernel)
  const double* __restrict__ U = cl.U;
  double* __restrict__ gt = cl.gt;
  const double tval = cl.t;
  const int ntl = (md.m + kFaceTile - 1) / kFaceTile;
  const int f = tl.y * kFaceTile + threadIdx.x;
  const double* __restrict__ lam = md.lam;
  const int clamp_on = md.clamp_on;
  const double clamp_min = md.clamp_min;
  double gt_part = 0.0;
  if (f < md.m) {
    int vid[3];
    double P[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      vid[c] = face_vertex(md, f, c);
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
      // <Lambda_v, B_v - U_v> of the three vertices, formed once per vertex by vjp_vertex_kernel
      wa = (__ldg(wvert + vid[0]) + __ldg(wvert + vid[1])) + __ldg(wvert + vid[2]);
      double L[3][K], Uv[3][K];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          L[c][k] = lam[(long)vid[c] * K + k];
          Uv[c][k] = U[(long)vid[c] * K + k];
        }
      }
      const double mt2 = -0.5 * tval;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        double lu = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) lu = fma(L[a][k] - L[b][k], Uv[a][k] - Uv[b][k], lu);
        // dl/dt = -<Lambda, L U> = -sum_c (cot_c / 2) lu_c = sum_c (dot_c / s / 2) lu_c
        if (CLAMP && clamp_on && -dot[c] * inv_s < clamp_min) {
          // a clamped corner holds cot = clamp_min: no term in dl/dV, clamp_min in dl/dt
          omega[c] = 0.0;
          if (gt) gt_part = fma(-0.5 * clamp_min, lu, gt_part);
        } else {
          omega[c] = mt2 * lu;
          if (gt) gt_part = fma(0.5 * dot[c] * inv_s, lu, gt_part);
        }
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

// K6a's per-vertex part: w_v = <Lambda_v, B_v - U_v> (the gradient of the face area's weight
// comes from these three per face), formed once per vertex instead of once per incident face. It
// goes to the solver's z vector, which no kernel reads between the adjoint solve and the next
// solve's initialisation.
template <int K>
__global__ void __launch_bounds__(256) vjp_vertex_kernel(const MeshDev* __restrict__ mds,
                                                         const CallDev* __restrict__ calls,
                                                         const int2* __restrict__ rtiles) {
  const int2 tl = rtiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const int v = tl.y * 256 + threadIdx.x;
  if (v >= md.n) return;
  const CallDev& cl = calls[tl.x];
  const double* __restrict__ Bsrc = cl.b_is_V ? cl.V : cl.B;
  double w = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k)
    w = fma(md.lam[(long)v * K + k], Bsrc[(long)v * cl.bstride + k] - cl.U[(long)v * K + k], w);
  md.z[v] = w;
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
  int e0, e1;
  inc_range(md, v, e0, e1);
  for (int e = e0; e < e1; ++e) {
    const int fc = __ldg(&md.inc[e].x);
    const double* src = md.gface + 9 * (long)inc_face(md, fc) + 3 * (fc & 3);
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

// ------------------------------------------------------------------------------- FP32 geometry
constexpr float kSliverSin2 = 1e-4f;  // the assembly's sliver test: sin^2 of the smallest corner

// usplit[v] = (hi of U_v (padded to 4), lo of U_v), lsplit[v] the same for Lambda, and
// wv[v] = <Lambda_v, B_v - U_v> in FP32 from the hi/lo parts (B_v - U_v may cancel).
template <int K>
__global__ void __launch_bounds__(256) vjp32_split_kernel(const MeshDev* __restrict__ mds,
                                                          const CallDev* __restrict__ calls,
                                                          const int2* __restrict__ rtiles) {
  const int2 tl = rtiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const int v = tl.y * 256 + threadIdx.x;
  if (v >= md.n) return;
  const CallDev& cl = calls[tl.x];
  const double* __restrict__ Bsrc = cl.b_is_V ? cl.V : cl.B;
  float uh[4] = {0.f, 0.f, 0.f, 0.f}, ul[4] = {0.f, 0.f, 0.f, 0.f};
  float lh[4] = {0.f, 0.f, 0.f, 0.f}, ll[4] = {0.f, 0.f, 0.f, 0.f};
  float w = 0.f;
#pragma unroll
  for (int c = 0; c < K; ++c) {
    float bh, bl;
    split_f64(__ldg(cl.U + (long)v * K + c), uh[c], ul[c]);
    split_f64(md.lam[(long)v * K + c], lh[c], ll[c]);
    split_f64(__ldg(Bsrc + (long)v * cl.bstride + c), bh, bl);
    w = fmaf(lh[c] + ll[c], (bh - uh[c]) + (bl - ul[c]), w);
  }
  float4* us = reinterpret_cast<float4*>(md.usplit) + 2 * (long)v;
  float4* ls = reinterpret_cast<float4*>(md.lsplit) + 2 * (long)v;
  us[0] = make_float4(uh[0], uh[1], uh[2], uh[3]);
  us[1] = make_float4(ul[0], ul[1], ul[2], ul[3]);
  ls[0] = make_float4(lh[0], lh[1], lh[2], lh[3]);
  ls[1] = make_float4(ll[0], ll[1], ll[2], ll[3]);
  md.wv[v] = w;
}

// The FP64 per-corner gradients of one face (the formula of vjp_face_kernel, mode 0), and its
// term of dl/dt; for slivers under FP32 geometry.
template <int K>
__device__ __noinline__ double face_grad64(const MeshDev& md, const CallDev& cl, const int (&vid)[3], double (&g)[9]) {
  const double* __restrict__ V = cl.V;
  const double* __restrict__ Bsrc = cl.b_is_V ? cl.V : cl.B;
  double P[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) P[c][d] = __ldg(V + 3 * (long)vid[c] + d);
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
  const double inv_s = rsqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
  double dot[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    dot[c] = dd[a][0] * dd[b][0] + dd[a][1] * dd[b][1] + dd[a][2] * dd[b][2];
  }
  double L[3][K], Uv[3][K], wa = 0.0, gt_part = 0.0;
  double omega[3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      L[c][k] = md.lam[(long)vid[c] * K + k];
      Uv[c][k] = __ldg(cl.U + (long)vid[c] * K + k);
      wa = fma(L[c][k], __ldg(Bsrc + (long)vid[c] * cl.bstride + k) - Uv[c][k], wa);
    }
  const double mt2 = -0.5 * cl.t;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    double lu = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) lu = fma(L[a][k] - L[b][k], Uv[a][k] - Uv[b][k], lu);
    if (md.clamp_on && -dot[c] * inv_s < md.clamp_min) {
      omega[c] = 0.0;
      gt_part = fma(-0.5 * md.clamp_min, lu, gt_part);
    } else {
      omega[c] = mt2 * lu;
      gt_part = fma(0.5 * dot[c] * inv_s, lu, gt_part);
    }
  }
  wa *= (1.0 / 3.0);
  const double Pv = -(omega[0] * dot[0] + omega[1] * dot[1] + omega[2] * dot[2]);
  const double coef = (0.5 * wa - Pv * inv_s * inv_s) * inv_s;
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
    for (int d = 0; d < 3; ++d) g[3 * c + d] = fma(coef, nxd[d], fma(dom, dd[c][d], -om * (dd[b][d] - dd[a][d])));
  }
  return gt_part;
}

__device__ __forceinline__ float hl_diff(float ha, float la, float hb, float lb) { return (ha - hb) + (la - lb); }

template <int K>
__global__ void __launch_bounds__(256, 3) vjp32_face_kernel(const MeshDev* __restrict__ mds,
                                                         const CallDev* __restrict__ calls,
                                                         const int2* __restrict__ ftiles) {
  __shared__ double sh[8];
  __shared__ int s_last;
  const int2 tl = ftiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const CallDev& cl = calls[tl.x];
  double* __restrict__ gt = cl.gt;
  const int ntl = (md.m + kFaceTile - 1) / kFaceTile;
  const int f = tl.y * kFaceTile + threadIdx.x;
  float gt_part = 0.f;
  double gt_part64 = 0.0;
  if (f < md.m) {
    int vid[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) vid[c] = face_vertex(md, f, c);
    const float4* __restrict__ vs = reinterpret_cast<const float4*>(md.vsplit);
    float4 ph[3], pl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ph[c] = __ldg(vs + 2 * (long)vid[c]);
      pl[c] = __ldg(vs + 2 * (long)vid[c] + 1);
    }
    // edges d_c = p_b - p_a for (a, b) = (c + 1, c + 2)
    float dd[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int a = (c + 1) % 3, b = (c + 2) % 3;
      dd[c][0] = hl_diff(ph[b].x, pl[b].x, ph[a].x, pl[a].x);
      dd[c][1] = hl_diff(ph[b].y, pl[b].y, ph[a].y, pl[a].y);
      dd[c][2] = hl_diff(ph[b].z, pl[b].z, ph[a].z, pl[a].z);
    }
    float N[3];
    N[0] = dd[1][1] * dd[2][2] - dd[1][2] * dd[2][1];
    N[1] = dd[1][2] * dd[2][0] - dd[1][0] * dd[2][2];
    N[2] = dd[1][0] * dd[2][1] - dd[1][1] * dd[2][0];
    const float s2 = N[0] * N[0] + N[1] * N[1] + N[2] * N[2];
    float e2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) e2[c] = dd[c][0] * dd[c][0] + dd[c][1] * dd[c][1] + dd[c][2] * dd[c][2];
    const float pmax = fmaxf(fmaxf(e2[1] * e2[2], e2[2] * e2[0]), e2[0] * e2[1]);
    float g[9];
    if (!(s2 >= kSliverSin2 * pmax) || !(s2 > 0.f) || !(pmax < 3.0e38f)) {
      double g64[9];
      gt_part64 = face_grad64<K>(md, cl, vid, g64);
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = (float)g64[i];
    } else {
      const float inv_s = rsqrtf(s2);
      float dot[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        dot[c] = dd[a][0] * dd[b][0] + dd[a][1] * dd[b][1] + dd[a][2] * dd[b][2];
      }
      const float4* __restrict__ us = reinterpret_cast<const float4*>(md.usplit);
      const float4* __restrict__ ls = reinterpret_cast<const float4*>(md.lsplit);
      float uh[3][4], ul[3][4], lh[3][4], ll[3][4];
      float wa = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 a = __ldg(us + 2 * (long)vid[c]), b = __ldg(us + 2 * (long)vid[c] + 1);
        const float4 x = __ldg(ls + 2 * (long)vid[c]), y = __ldg(ls + 2 * (long)vid[c] + 1);
        uh[c][0] = a.x; uh[c][1] = a.y; uh[c][2] = a.z; uh[c][3] = a.w;
        ul[c][0] = b.x; ul[c][1] = b.y; ul[c][2] = b.z; ul[c][3] = b.w;
        lh[c][0] = x.x; lh[c][1] = x.y; lh[c][2] = x.z; lh[c][3] = x.w;
        ll[c][0] = y.x; ll[c][1] = y.y; ll[c][2] = y.z; ll[c][3] = y.w;
        wa += __ldg(md.wv + vid[c]);
      }
      float th, tl32;
      split_f64(cl.t, th, tl32);
      const float mt2 = -0.5f * (th + tl32);
      const bool clamp_on = md.clamp_on != 0;
      float cmin = 0.f;
      if (clamp_on) {
        float ch, cl2;
        split_f64(md.clamp_min, ch, cl2);
        cmin = ch + cl2;
      }
      float omega[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        float lu = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k)
          lu = fmaf(hl_diff(lh[a][k], ll[a][k], lh[b][k], ll[b][k]), hl_diff(uh[a][k], ul[a][k], uh[b][k], ul[b][k]),
                    lu);
        if (clamp_on && -dot[c] * inv_s < cmin) {
          omega[c] = 0.f;
          gt_part = fmaf(-0.5f * cmin, lu, gt_part);
        } else {
          omega[c] = mt2 * lu;
          gt_part = fmaf(0.5f * dot[c] * inv_s, lu, gt_part);
        }
      }
      wa *= (1.0f / 3.0f);
      const float Pv = -(omega[0] * dot[0] + omega[1] * dot[1] + omega[2] * dot[2]);
      const float coef = (0.5f * wa - Pv * inv_s * inv_s) * inv_s;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        const float om = omega[c] * inv_s;
        const float dom = (omega[a] - omega[b]) * inv_s;
        float nxd[3];
        nxd[0] = N[1] * dd[c][2] - N[2] * dd[c][1];
        nxd[1] = N[2] * dd[c][0] - N[0] * dd[c][2];
        nxd[2] = N[0] * dd[c][1] - N[1] * dd[c][0];
#pragma unroll
        for (int d = 0; d < 3; ++d) g[3 * c + d] = fmaf(coef, nxd[d], fmaf(dom, dd[c][d], -om * (dd[b][d] - dd[a][d])));
      }
    }
    float4* out = reinterpret_cast<float4*>(md.gface) + 3 * (long)f;
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = make_float4(g[3 * c], g[3 * c + 1], g[3 * c + 2], 0.f);
  }
  if (gt == nullptr) return;
  // dl/dt: FP32 per thread (FP64 for slivers), the CTA's partial in FP64, the last CTA adds the
  // partials in order
  double part = gt_part64;
  {
    float x = gt_part;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = part + f32_to_f64(x);
  }
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
__global__ void __launch_bounds__(256) vjp32_gather_kernel(const MeshDev* __restrict__ mds,
                                                           const CallDev* __restrict__ calls,
                                                           const int2* __restrict__ rtiles) {
  const int2 tl = rtiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const int v = tl.y * 256 + threadIdx.x;
  if (v >= md.n) return;
  const int b_is_V = calls[tl.x].b_is_V;
  double* __restrict__ gV = calls[tl.x].gV;
  double* __restrict__ gB = calls[tl.x].gB;
  const float4* __restrict__ gf = reinterpret_cast<const float4*>(md.gface);
  float g0 = 0.f, g1 = 0.f, g2 = 0.f;
  int e0, e1;
  inc_range(md, v, e0, e1);
  for (int e = e0; e < e1; ++e) {
    const int fc = __ldg(&md.inc[e].x);
    const float4 x = __ldg(gf + 3 * (long)inc_face(md, fc) + (fc & 3));
    g0 += x.x;
    g1 += x.y;
    g2 += x.z;
  }
  double o0 = f32_to_f64(g0), o1 = f32_to_f64(g1), o2 = f32_to_f64(g2);
  if (b_is_V || gB) {
    const double mass = md.M[v];
    if (b_is_V) {
      o0 = fma(mass, md.lam[(long)v * K + 0], o0);
      o1 = fma(mass, md.lam[(long)v * K + 1], o1);
      o2 = fma(mass, md.lam[(long)v * K + 2], o2);
    }
    if (gB) {
#pragma unroll
      for (int k = 0; k < K; ++k) gB[(long)v * K + k] = mass * md.lam[(long)v * K + k];
    }
  }
  gV[3 * (long)v + 0] = o0;
  gV[3 * (long)v + 1] = o1;
  gV[3 * (long)v + 2] = o2;
}

template <int K>
cudaError_t vjp32_k(Group& g, cudaStream_t st) {
  cudaError_t e;
  {
    IG_PROF("vjp_split32", st);
    vjp32_split_kernel<K><<<g.nrow_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.row_tiles);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    IG_PROF("vjp_face32", st);
    vjp32_face_kernel<K><<<g.nface_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.face_tiles);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    IG_PROF("vjp_gather32", st);
    vjp32_gather_kernel<K><<<g.nrow_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.row_tiles);
  }
  return cudaGetLastError();
}

template <int K>
cudaError_t vjp_k(Group& g, int mode, cudaStream_t st) {
  if (mode != 2) {
    IG_PROF("vjp_vertex", st);
    vjp_vertex_kernel<K><<<g.nrow_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.row_tiles);
  }
  {
    IG_PROF("vjp_face", st);
    const bool cl = group_any_clamp(g);
    if (mode == 0 && cl) vjp_face_kernel<K, 0, true><<<g.nface_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.face_tiles);
    else if (mode == 0) vjp_face_kernel<K, 0, false><<<g.nface_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.face_tiles);
    else if (mode == 1 && cl)
      vjp_face_kernel<K, 1, true><<<g.nface_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.face_tiles);
    else if (mode == 1) vjp_face_kernel<K, 1, false><<<g.nface_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.face_tiles);
    else vjp_face_kernel<K, 2, false><<<g.nface_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.face_tiles);
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

cudaError_t launch_vjp(Group& g, int k, cudaStream_t st, int mode, int geom32) {
  if (mode == 2) return vjp_k<1>(g, 2, st);
  if (mode == 0 && geom32) {
    switch (k) {
      case 1: return vjp32_k<1>(g, st);
      case 2: return vjp32_k<2>(g, st);
      case 3: return vjp32_k<3>(g, st);
      case 4: return vjp32_k<4>(g, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (k) {
    case 1: return vjp_k<1>(g, mode, st);
    case 2: return vjp_k<2>(g, mode, st);
    case 3: return vjp_k<3>(g, mode, st);
    case 4: return vjp_k<4>(g, mode, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ig
