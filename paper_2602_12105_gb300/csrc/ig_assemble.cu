// ig_assemble.cu -- assembly of A = M(V) + t L(V) on the fixed pattern (§7.1: the cotangent
// Laplacian L(v) and the diagonal mass M(v) are recomputed from the positions every step).
//
// K1 (face-parallel): for face (p0, p1, p2) let d_c be the edge opposite corner c, oriented
//   d_0 = p2 - p1, d_1 = p0 - p2, d_2 = p1 - p0, and N = d_1 x d_2 (twice the area vector,
//   s = |N|). The cotangent of corner c is cot_c = -(d_{c+1} . d_{c+2}) / s. K1 stores per face
//   w_c = t cot_c / 2 (the weight of the edge opposite c in t L) and s / 6 (area / 3).
// K2 (row-parallel, atomic-free): each row gathers the faces around its vertex from the
//   incidence list (sorted by face, so the summation order is fixed): the edge to the next
//   corner receives -w of the previous corner, the edge to the previous corner -w of the next
//   one, the diagonal the sum of both, the mass area/3. It writes A = M + tL, M, 1/A_ii and, in
//   mixed precision, FP32 copies of A and 1/A_ii.
//
// FP64 arithmetic is the scarce resource on this part (2 FP64 FMA per clock per SM), so the
// kernels avoid FP64 compares (validity is tested on the bit patterns) and fold t/2 into K1.
//
// FP32 face geometry (mixed precision with FP32 cotangents): a vertex pass splits each position
// into hi/lo floats (integer instructions only); K1 forms the edges as (hi_b - hi_a) + (lo_b - lo_a),
// which keeps FP32 relative accuracy however close the vertices are, and computes cot and area in
// FP32. A face whose smallest corner has sin(theta) < 1e-2 (a sliver: the FP32 cotangent of that
// corner would lose up to 1/sin(theta) of its accuracy to the cross product) is computed in FP64
// from the FP64 positions instead. K2 then sums the FP32 weights into the FP32 operator A32, which
// is the operator of this mode (its values are exact in FP64 too: every residual uses them).
#include "ig_f32.cuh"
#include "ig_internal.cuh"

namespace ig {

namespace {

// True when x is finite and > 0 (x is known to be >= 0 or NaN): integer test, no FP64 op.
__device__ __forceinline__ bool positive_finite(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && (b & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}

// CLAMP: some mesh of the group clamps its cotangents (the check is compiled out otherwise: this
// kernel is bound by FP64 instructions).
template <bool CLAMP>
__global__ void __launch_bounds__(256) face_kernel(const MeshDev* __restrict__ mds, const CallDev* __restrict__ calls,
                                                   const int2* __restrict__ ftiles) {
  const int2 tl = ftiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const int f = tl.y * 256 + threadIdx.x;
  if (f >= md.m) return;
  const double* __restrict__ V = calls[tl.x].V;
  const double half_t = 0.5 * calls[tl.x].t;
  double* __restrict__ facew = md.facew;
  int* err = md.err;
  const int i0 = face_vertex(md, f, 0), i1 = face_vertex(md, f, 1), i2 = face_vertex(md, f, 2);
  double p0[3], p1[3], p2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    p0[d] = __ldg(V + 3 * (long)i0 + d);
    p1[d] = __ldg(V + 3 * (long)i1 + d);
    p2[d] = __ldg(V + 3 * (long)i2 + d);
  }
  double d0[3], d1[3], d2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    d0[d] = p2[d] - p1[d];
    d1[d] = p0[d] - p2[d];
    d2[d] = p1[d] - p0[d];
  }
  const double nx = d1[1] * d2[2] - d1[2] * d2[1];
  const double ny = d1[2] * d2[0] - d1[0] * d2[2];
  const double nz = d1[0] * d2[1] - d1[1] * d2[0];
  const double s2 = nx * nx + ny * ny + nz * nz;
  double wx, wy, wz, ww;  // the three corner weights and the face area / 3
  if (!positive_finite(s2)) {
    const long long b = __double_as_longlong(s2);
    atomicOr(err, (b & 0x7ff0000000000000ll) == 0x7ff0000000000000ll ? kErrNonfinite : kErrDegenerate);
    wx = wy = wz = ww = 0.0;
  } else {
    const double inv_s = rsqrt(s2);
    const double h = -half_t * inv_s;
    wx = h * (d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2]);
    wy = h * (d2[0] * d0[0] + d2[1] * d0[1] + d2[2] * d0[2]);
    wz = h * (d0[0] * d1[0] + d0[1] * d1[1] + d0[2] * d1[2]);
    ww = s2 * inv_s * (1.0 / 6.0);
    if (CLAMP && md.clamp_on) {  // w_c = (t/2) cot_c >= (t/2) clamp_min
      const double wmin = half_t * md.clamp_min;
      wx = fmax(wx, wmin);
      wy = fmax(wy, wmin);
      wz = fmax(wz, wmin);
    }
  }
  double2* out = reinterpret_cast<double2*>(facew + 4 * (long)f);
  out[0] = make_double2(wx, wy);
  out[1] = make_double2(wz, ww);
}

// sin^2 of the smallest corner below this: the face is a sliver and is computed in FP64.
constexpr float kSliverSin2 = 1e-4f;

// Positions split into hi/lo floats: vsplit[v] = (hx, hy, hz, 0, lx, ly, lz, 0).
__global__ void __launch_bounds__(256) split_v_kernel(const MeshDev* __restrict__ mds,
                                                      const CallDev* __restrict__ calls,
                                                      const int2* __restrict__ rtiles) {
  const int2 tl = rtiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const int v = tl.y * 256 + threadIdx.x;
  if (v >= md.n) return;
  const double* __restrict__ V = calls[tl.x].V;
  float h[3], l[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) split_f64(__ldg(V + 3 * (long)v + d), h[d], l[d]);
  float4* out = reinterpret_cast<float4*>(md.vsplit) + 2 * (long)v;
  out[0] = make_float4(h[0], h[1], h[2], 0.f);
  out[1] = make_float4(l[0], l[1], l[2], 0.f);
}

// The FP64 weights of one face (as face_kernel), rounded to float; flags a degenerate or
// non-finite face.
__device__ __noinline__ float4 face_weights64(const double* __restrict__ V, int i0, int i1, int i2, double half_t,
                                              int* err, int clamp_on, double clamp_min) {
  double p0[3], p1[3], p2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    p0[d] = __ldg(V + 3 * (long)i0 + d);
    p1[d] = __ldg(V + 3 * (long)i1 + d);
    p2[d] = __ldg(V + 3 * (long)i2 + d);
  }
  double d0[3], d1[3], d2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    d0[d] = p2[d] - p1[d];
    d1[d] = p0[d] - p2[d];
    d2[d] = p1[d] - p0[d];
  }
  const double nx = d1[1] * d2[2] - d1[2] * d2[1];
  const double ny = d1[2] * d2[0] - d1[0] * d2[2];
  const double nz = d1[0] * d2[1] - d1[1] * d2[0];
  const double s2 = nx * nx + ny * ny + nz * nz;
  if (!positive_finite(s2)) {
    const long long b = __double_as_longlong(s2);
    atomicOr(err, (b & 0x7ff0000000000000ll) == 0x7ff0000000000000ll ? kErrNonfinite : kErrDegenerate);
    return make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const double inv_s = rsqrt(s2);
  const double h = -half_t * inv_s;
  double w0 = h * (d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2]);
  double w1 = h * (d2[0] * d0[0] + d2[1] * d0[1] + d2[2] * d0[2]);
  double w2 = h * (d0[0] * d1[0] + d0[1] * d1[1] + d0[2] * d1[2]);
  if (clamp_on) {
    const double wmin = half_t * clamp_min;
    w0 = fmax(w0, wmin);
    w1 = fmax(w1, wmin);
    w2 = fmax(w2, wmin);
  }
  return make_float4((float)w0, (float)w1, (float)w2, (float)(s2 * inv_s * (1.0 / 6.0)));
}

// K1 with FP32 geometry: per face the float weights (t cot_c / 2, area / 3) into facew viewed as
// [m][4] float.
__global__ void __launch_bounds__(256) face32_kernel(const MeshDev* __restrict__ mds,
                                                     const CallDev* __restrict__ calls,
                                                     const int2* __restrict__ ftiles) {
  const int2 tl = ftiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const int f = tl.y * 256 + threadIdx.x;
  if (f >= md.m) return;
  const int i0 = face_vertex(md, f, 0), i1 = face_vertex(md, f, 1), i2 = face_vertex(md, f, 2);
  const float4* __restrict__ vs = reinterpret_cast<const float4*>(md.vsplit);
  const float4 h0 = __ldg(vs + 2 * (long)i0), l0 = __ldg(vs + 2 * (long)i0 + 1);
  const float4 h1 = __ldg(vs + 2 * (long)i1), l1 = __ldg(vs + 2 * (long)i1 + 1);
  const float4 h2 = __ldg(vs + 2 * (long)i2), l2 = __ldg(vs + 2 * (long)i2 + 1);
  // d0 = p2 - p1, d1 = p0 - p2, d2 = p1 - p0
  const float d0x = (h2.x - h1.x) + (l2.x - l1.x), d0y = (h2.y - h1.y) + (l2.y - l1.y),
              d0z = (h2.z - h1.z) + (l2.z - l1.z);
  const float d1x = (h0.x - h2.x) + (l0.x - l2.x), d1y = (h0.y - h2.y) + (l0.y - l2.y),
              d1z = (h0.z - h2.z) + (l0.z - l2.z);
  const float d2x = (h1.x - h0.x) + (l1.x - l0.x), d2y = (h1.y - h0.y) + (l1.y - l0.y),
              d2z = (h1.z - h0.z) + (l1.z - l0.z);
  const float nx = d1y * d2z - d1z * d2y, ny = d1z * d2x - d1x * d2z, nz = d1x * d2y - d1y * d2x;
  const float s2 = nx * nx + ny * ny + nz * nz;
  const float e0 = d0x * d0x + d0y * d0y + d0z * d0z, e1 = d1x * d1x + d1y * d1y + d1z * d1z,
              e2 = d2x * d2x + d2y * d2y + d2z * d2z;
  // sin^2 of the smallest corner = s^2 / (product of the two longest squared edges)
  const float pmax = fmaxf(fmaxf(e1 * e2, e2 * e0), e0 * e1);
  float4 w;
  if (!(s2 >= kSliverSin2 * pmax) || !(s2 > 0.f) || !(pmax < 3.0e38f)) {
    w = face_weights64(calls[tl.x].V, i0, i1, i2, 0.5 * calls[tl.x].t, md.err, md.clamp_on, md.clamp_min);
  } else {
    float th, tl32;
    split_f64(calls[tl.x].t, th, tl32);  // t as a float without an FP64 conversion instruction
    const float inv_s = rsqrtf(s2);
    const float half_t = 0.5f * (th + tl32);
    const float h = -half_t * inv_s;
    w.x = h * (d1x * d2x + d1y * d2y + d1z * d2z);
    w.y = h * (d2x * d0x + d2y * d0y + d2z * d0z);
    w.z = h * (d0x * d1x + d0y * d1y + d0z * d1z);
    w.w = s2 * inv_s * (1.0f / 6.0f);
    if (md.clamp_on) {
      float ch, cl;
      split_f64(md.clamp_min, ch, cl);
      const float wmin = half_t * (ch + cl);
      w.x = fmaxf(w.x, wmin);
      w.y = fmaxf(w.y, wmin);
      w.z = fmaxf(w.z, wmin);
    }
  }
  reinterpret_cast<float4*>(md.facew)[f] = w;
}

constexpr int kSmemSlots = 16;  // rows up to this length accumulate in shared memory

// K2 with FP32 geometry: the FP32 operator A32 (sliced layout), the mass M (the float sum, stored
// exactly in FP64) and the FP32 inverse diagonal. The summation order is fixed (the incidence is
// sorted by face), so the two rows that share an edge add its two weights in the same order and
// A32 is exactly symmetric.
__global__ void __launch_bounds__(256) row32_kernel(const MeshDev* __restrict__ mds, const int2* __restrict__ rtiles) {
  __shared__ float acc[kSmemSlots][256];
  const int2 tl = rtiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const int v = tl.y * 256 + threadIdx.x;
  if (v >= md.n) return;
  const int r0 = __ldg(md.rowptr + v);
  const int len = __ldg(md.rowptr + v + 1) - r0;
  int dslot = __ldg(md.diagpos + v) - r0;
#ifdef IG_CHECK
  if (!IG_IN_RANGE(dslot, len, md.err)) dslot = 0;
#endif
  const int sl = v >> 5;
  const int sbase = __ldg(md.sell_ptr + sl) + (v & 31);
  const int width = (__ldg(md.sell_ptr + sl + 1) - __ldg(md.sell_ptr + sl)) >> 5;
  const bool in_smem = len <= kSmemSlots;
  float* gA = md.A32;
  if (in_smem) {
    for (int j = 0; j < len; ++j) acc[j][threadIdx.x] = 0.f;
  } else {
    for (int j = 0; j < len; ++j) gA[sbase + 32 * j] = 0.f;
  }
  float mass = 0.f, diag = 0.f;
  const float4* __restrict__ fw4 = reinterpret_cast<const float4*>(md.facew);
  int e0, e1;
  inc_range(md, v, e0, e1);
  for (int e = e0; e < e1; ++e) {
    const int2 ic = __ldg(md.inc + e);
    const int f = inc_face(md, ic.x), c = ic.x & 3;
    const float4 w = __ldg(fw4 + f);
    const float w_next = (c == 0) ? w.z : (c == 1 ? w.x : w.y);
    const float w_prev = (c == 0) ? w.y : (c == 1 ? w.z : w.x);
    const int sn = ic.y & 0xffff, sp = ic.y >> 16;
#ifdef IG_CHECK
    if (!IG_IN_RANGE(sn, len, md.err) || !IG_IN_RANGE(sp, len, md.err)) continue;
#endif
    if (in_smem) {
      acc[sn][threadIdx.x] -= w_next;
      acc[sp][threadIdx.x] -= w_prev;
    } else {
      gA[sbase + 32 * sn] -= w_next;
      gA[sbase + 32 * sp] -= w_prev;
    }
    diag += w_next + w_prev;
    mass += w.w;
  }
  const float aii = mass + diag;
  if (in_smem) {
    acc[dslot][threadIdx.x] = aii;
    for (int j = 0; j < len; ++j) gA[sbase + 32 * j] = acc[j][threadIdx.x];
  } else {
    gA[sbase + 32 * dslot] = aii;
  }
  for (int j = len; j < width; ++j) gA[sbase + 32 * j] = 0.f;
  md.M[v] = f32_to_f64(mass);
  md.Dinv32[v] = 1.0f / aii;
}

// Values of row v go to the sliced layout: slot j at sell_ptr[v/32] + 32 j + v%32; slots between
// the row's length and the slice width are written as 0.
__global__ void __launch_bounds__(256) row_kernel(const MeshDev* __restrict__ mds, const int2* __restrict__ rtiles,
                                                  int mixed) {
  __shared__ double acc[kSmemSlots][256];
  const int2 tl = rtiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const int v = tl.y * 256 + threadIdx.x;
  if (v >= md.n) return;
  const int r0 = __ldg(md.rowptr + v);
  const int len = __ldg(md.rowptr + v + 1) - r0;
  int dslot = __ldg(md.diagpos + v) - r0;
#ifdef IG_CHECK
  if (!IG_IN_RANGE(dslot, len, md.err)) dslot = 0;
#endif
  const int sl = v >> 5;
  const int sbase = __ldg(md.sell_ptr + sl) + (v & 31);
  const int width = (__ldg(md.sell_ptr + sl + 1) - __ldg(md.sell_ptr + sl)) >> 5;
  const bool in_smem = len <= kSmemSlots;
  double* gA = md.A;
  if (in_smem) {
    for (int j = 0; j < len; ++j) acc[j][threadIdx.x] = 0.0;
  } else {
    for (int j = 0; j < len; ++j) gA[sbase + 32 * j] = 0.0;
  }
  double mass = 0.0, diag = 0.0;
  int e0, e1;
  inc_range(md, v, e0, e1);
  for (int e = e0; e < e1; ++e) {
    const int2 ic = __ldg(md.inc + e);
    const int f = inc_face(md, ic.x), c = ic.x & 3;
    const double2* fw = reinterpret_cast<const double2*>(md.facew + 4 * (long)f);
    const double2 a = __ldg(fw), b = __ldg(fw + 1);
    // corner c+2 is opposite the edge (v, next); corner c+1 is opposite the edge (v, prev)
    const double w_next = (c == 0) ? b.x : (c == 1 ? a.x : a.y);
    const double w_prev = (c == 0) ? a.y : (c == 1 ? b.x : a.x);
    const int sn = ic.y & 0xffff, sp = ic.y >> 16;
#ifdef IG_CHECK
    if (!IG_IN_RANGE(sn, len, md.err) || !IG_IN_RANGE(sp, len, md.err)) continue;
#endif
    if (in_smem) {
      acc[sn][threadIdx.x] -= w_next;
      acc[sp][threadIdx.x] -= w_prev;
    } else {
      gA[sbase + 32 * sn] -= w_next;
      gA[sbase + 32 * sp] -= w_prev;
    }
    diag += w_next + w_prev;
    mass += b.y;
  }
  const double aii = mass + diag;
  const double dinv = 1.0 / aii;
  // the FP32 copies round to nearest with integer instructions (f64_to_f32_rn), not the
  // conversion instruction, which issues at the FP64 rate
  if (in_smem) {
    acc[dslot][threadIdx.x] = aii;
    for (int j = 0; j < len; ++j) {
      const double x = acc[j][threadIdx.x];
      gA[sbase + 32 * j] = x;
      if (mixed) md.A32[sbase + 32 * j] = f64_to_f32_rn(x);
    }
  } else {
    gA[sbase + 32 * dslot] = aii;
    if (mixed)
      for (int j = 0; j < len; ++j) md.A32[sbase + 32 * j] = f64_to_f32_rn(gA[sbase + 32 * j]);
  }
  for (int j = len; j < width; ++j) {
    gA[sbase + 32 * j] = 0.0;
    if (mixed) md.A32[sbase + 32 * j] = 0.f;
  }
  md.M[v] = mass;
  md.Dinv[v] = dinv;
  if (mixed) md.Dinv32[v] = f64_to_f32_rn(dinv);
}

// Copy of A in CSR order (the order of ig_mesh_pattern); with FP32 geometry the FP32 operator.
__global__ void __launch_bounds__(256) operator_csr_kernel(MeshDev md, double* __restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= md.n) return;
  const int r0 = md.rowptr[v], len = md.rowptr[v + 1] - r0;
  const int sbase = md.sell_ptr[v >> 5] + (v & 31);
  for (int j = 0; j < len; ++j)
    out[r0 + j] = md.geom32 ? f32_to_f64(md.A32[sbase + 32 * j]) : md.A[sbase + 32 * j];
}

// The FP32 operator (mixed precision) in CSR order.
__global__ void __launch_bounds__(256) operator32_csr_kernel(MeshDev md, float* __restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= md.n) return;
  const int r0 = md.rowptr[v], len = md.rowptr[v + 1] - r0;
  const int sbase = md.sell_ptr[v >> 5] + (v & 31);
  for (int j = 0; j < len; ++j) out[r0 + j] = md.A32[sbase + 32 * j];
}

}  // namespace

cudaError_t launch_assemble(Group& g, int mode, cudaStream_t st) {
  cudaError_t e;
  if (mode == 2) {
    {
      IG_PROF("assemble_split32", st);
      split_v_kernel<<<g.nrow_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.row_tiles);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
      IG_PROF("assemble_face32", st);
      face32_kernel<<<g.nface_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.face_tiles);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
      IG_PROF("assemble_rows32", st);
      row32_kernel<<<g.nrow_tiles, 256, 0, st>>>(g.mds, g.row_tiles);
    }
    return cudaGetLastError();
  }
  {
    IG_PROF("assemble_face", st);
    if (group_any_clamp(g)) face_kernel<true><<<g.nface_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.face_tiles);
    else face_kernel<false><<<g.nface_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.face_tiles);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    IG_PROF("assemble_rows", st);
    row_kernel<<<g.nrow_tiles, 256, 0, st>>>(g.mds, g.row_tiles, mode);
  }
  return cudaGetLastError();
}

cudaError_t launch_operator32_csr(const MeshDev& md, float* Acsr, cudaStream_t st) {
  operator32_csr_kernel<<<(md.n + 255) / 256, 256, 0, st>>>(md, Acsr);
  return cudaGetLastError();
}

cudaError_t launch_operator_csr(const MeshDev& md, double* Acsr, cudaStream_t st) {
  operator_csr_kernel<<<(md.n + 255) / 256, 256, 0, st>>>(md, Acsr);
  return cudaGetLastError();
}

}  // namespace ig
