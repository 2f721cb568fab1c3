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
#include "ig_internal.cuh"

namespace ig {

namespace {

// True when x is finite and > 0 (x is known to be >= 0 or NaN): integer test, no FP64 op.
__device__ __forceinline__ bool positive_finite(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && (b & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}

__global__ void __launch_bounds__(256) face_kernel(const MeshDev* __restrict__ mds, const CallDev* __restrict__ calls,
                                                   const int2* __restrict__ ftiles) {
  const int2 tl = ftiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const int f = tl.y * 256 + threadIdx.x;
  if (f >= md.m) return;
  const double* __restrict__ V = calls[tl.x].V;
  const double half_t = 0.5 * calls[tl.x].t;
  const int* __restrict__ F = md.F;
  double* __restrict__ facew = md.facew;
  int* err = md.err;
  const int i0 = __ldg(F + 3 * f), i1 = __ldg(F + 3 * f + 1), i2 = __ldg(F + 3 * f + 2);
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
  double4 w;
  if (!positive_finite(s2)) {
    const long long b = __double_as_longlong(s2);
    atomicOr(err, (b & 0x7ff0000000000000ll) == 0x7ff0000000000000ll ? kErrNonfinite : kErrDegenerate);
    w = make_double4(0.0, 0.0, 0.0, 0.0);
  } else {
    const double inv_s = rsqrt(s2);
    const double h = -half_t * inv_s;
    w.x = h * (d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2]);
    w.y = h * (d2[0] * d0[0] + d2[1] * d0[1] + d2[2] * d0[2]);
    w.z = h * (d0[0] * d1[0] + d0[1] * d1[1] + d0[2] * d1[2]);
    w.w = s2 * inv_s * (1.0 / 6.0);
  }
  double2* out = reinterpret_cast<double2*>(facew + 4 * (long)f);
  out[0] = make_double2(w.x, w.y);
  out[1] = make_double2(w.z, w.w);
}

constexpr int kSmemSlots = 16;  // rows up to this length accumulate in shared memory

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
  const int dslot = __ldg(md.diagpos + v) - r0;
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
  const int e0 = __ldg(md.incptr + v), e1 = __ldg(md.incptr + v + 1);
  for (int e = e0; e < e1; ++e) {
    const int2 ic = __ldg(md.inc + e);
    const int f = ic.x >> 2, c = ic.x & 3;
    const double2* fw = reinterpret_cast<const double2*>(md.facew + 4 * (long)f);
    const double2 a = __ldg(fw), b = __ldg(fw + 1);
    // corner c+2 is opposite the edge (v, next); corner c+1 is opposite the edge (v, prev)
    const double w_next = (c == 0) ? b.x : (c == 1 ? a.x : a.y);
    const double w_prev = (c == 0) ? a.y : (c == 1 ? b.x : a.x);
    const int sn = ic.y & 0xffff, sp = ic.y >> 16;
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
  if (in_smem) {
    acc[dslot][threadIdx.x] = aii;
    for (int j = 0; j < len; ++j) {
      const double x = acc[j][threadIdx.x];
      gA[sbase + 32 * j] = x;
      if (mixed) md.A32[sbase + 32 * j] = (float)x;
    }
  } else {
    gA[sbase + 32 * dslot] = aii;
    if (mixed)
      for (int j = 0; j < len; ++j) md.A32[sbase + 32 * j] = (float)gA[sbase + 32 * j];
  }
  for (int j = len; j < width; ++j) {
    gA[sbase + 32 * j] = 0.0;
    if (mixed) md.A32[sbase + 32 * j] = 0.f;
  }
  md.M[v] = mass;
  md.Dinv[v] = dinv;
  if (mixed) md.Dinv32[v] = (float)dinv;
}

// Copy of A in CSR order (the order of ig_mesh_pattern).
__global__ void __launch_bounds__(256) operator_csr_kernel(MeshDev md, double* __restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= md.n) return;
  const int r0 = md.rowptr[v], len = md.rowptr[v + 1] - r0;
  const int sbase = md.sell_ptr[v >> 5] + (v & 31);
  for (int j = 0; j < len; ++j) out[r0 + j] = md.A[sbase + 32 * j];
}

}  // namespace

cudaError_t launch_assemble(Group& g, int mixed, cudaStream_t st) {
  {
    IG_PROF("assemble_face", st);
    face_kernel<<<g.nface_tiles, 256, 0, st>>>(g.mds, g.calls_dev, g.face_tiles);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    IG_PROF("assemble_rows", st);
    row_kernel<<<g.nrow_tiles, 256, 0, st>>>(g.mds, g.row_tiles, mixed);
  }
  return cudaGetLastError();
}

cudaError_t launch_operator_csr(const MeshDev& md, double* Acsr, cudaStream_t st) {
  operator_csr_kernel<<<(md.n + 255) / 256, 256, 0, st>>>(md, Acsr);
  return cudaGetLastError();
}

}  // namespace ig
