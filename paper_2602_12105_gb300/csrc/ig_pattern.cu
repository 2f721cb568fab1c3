// ig_pattern.cu -- topology-only structures, built once per mesh on the device.
//
// The paper keeps the sparsity pattern of M and L fixed while v changes and reuses what depends
// on it alone (§7.1). Here that is the CSR pattern of L (one row per vertex: the vertex itself
// and its edge neighbours, sorted) and a vertex -> (face, corner) incidence list that lets the
// assembly and the gradient gather per vertex instead of scattering per face with atomics.
//
// Steps (all on the device; only the two totals travel to the host):
//   count : per face, validate indices and count vertex-face incidences
//   scan  : incptr = exclusive scan of the counts
//   fill  : write face*4+corner into each vertex's incidence range (arbitrary order)
//   rows  : per vertex, sort its incidences, gather neighbour ids, sort + deduplicate -> row length
//   scan  : rowptr = exclusive scan of the row lengths
//   cols  : per vertex, write its columns, the diagonal position and the two row slots every
//           incidence contributes to
#include "ig_internal.cuh"

namespace ig {

namespace {

constexpr int kScanBlock = 1024;  // elements per CTA of the scan (256 threads x 4)

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive scan of in[0, count) (+ a virtual 0 at index count, so out[count] = total) in
// blocks of kScanBlock; block totals go to sums.
__global__ void __launch_bounds__(256) scan_block_kernel(const int* __restrict__ in, int* __restrict__ out,
                                                         int count, int total_len, int* __restrict__ sums) {
  __shared__ int warp_tot[8];
  const int base = blockIdx.x * kScanBlock + threadIdx.x * 4;
  int v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = (base + j < count) ? in[base + j] : 0;
  const int tsum = v[0] + v[1] + v[2] + v[3];
  const int incl = warp_incl_scan(tsum);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  int woff = 0;
  for (int w = 0; w < warp; ++w) woff += warp_tot[w];
  int run = woff + incl - tsum;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (base + j < total_len) out[base + j] = run;
    run += v[j];
  }
  if (threadIdx.x == 255) sums[blockIdx.x] = woff + incl;
}

__global__ void scan_add_kernel(int* __restrict__ out, int total_len, const int* __restrict__ offs) {
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  const int add = offs[blockIdx.x];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int e = i + j * 256;
    if (e < total_len) out[e] += add;
  }
}

}  // namespace

size_t scan_scratch_ints(int count) {
  size_t total = 0;
  long len = (long)count + 1;
  while (len > 1) {
    long nb = (len + kScanBlock - 1) / kScanBlock;
    total += 2 * (size_t)nb + 2;
    len = nb;
  }
  return total + 4;
}

// out[0..count] = exclusive scan of in[0..count) with out[count] = total. If total_out_dev is
// non-null the total is also copied there.
cudaError_t exclusive_scan_int(const int* in, int* out, int count, int* total_out_dev, int* scratch,
                               size_t scratch_ints, cudaStream_t st) {
  const int total_len = count + 1;
  const int nb = (total_len + kScanBlock - 1) / kScanBlock;
  if ((size_t)(2 * nb + 2) > scratch_ints) return cudaErrorInvalidValue;
  int* sums = scratch;
  int* sums_scan = scratch + nb + 1;
  scan_block_kernel<<<nb, 256, 0, st>>>(in, out, count, total_len, sums);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (nb > 1) {
    e = exclusive_scan_int(sums, sums_scan, nb, nullptr, scratch + 2 * nb + 2, scratch_ints - (2 * nb + 2), st);
    if (e != cudaSuccess) return e;
    scan_add_kernel<<<nb, 256, 0, st>>>(out, total_len, sums_scan);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (total_out_dev) e = cudaMemcpyAsync(total_out_dev, out + count, sizeof(int), cudaMemcpyDeviceToDevice, st);
  return e;
}

// ------------------------------------------------------------------------------- K0 kernels
namespace {

__global__ void __launch_bounds__(256) count_kernel(const int* __restrict__ F, int m, int n, int* __restrict__ deg,
                                                    int* __restrict__ err) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= m) return;
  const int a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
  if ((unsigned)a >= (unsigned)n || (unsigned)b >= (unsigned)n || (unsigned)c >= (unsigned)n) {
    atomicOr(err, kErrIndex);
    return;
  }
  if (a == b || b == c || a == c) {
    atomicOr(err, kErrRepeated);
    return;
  }
  atomicAdd(&deg[a], 1);
  atomicAdd(&deg[b], 1);
  atomicAdd(&deg[c], 1);
}

__global__ void __launch_bounds__(256) fill_kernel(const int* __restrict__ F, int m, const int* __restrict__ incptr,
                                                   int* __restrict__ fill, int* __restrict__ inc_fc) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= m) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int v = F[3 * f + c];
    const int pos = incptr[v] + atomicAdd(&fill[v], 1);
    inc_fc[pos] = f * 4 + c;
  }
}

__device__ __forceinline__ void insertion_sort(int* a, int len) {
  for (int i = 1; i < len; ++i) {
    const int x = a[i];
    int j = i - 1;
    while (j >= 0 && a[j] > x) {
      a[j + 1] = a[j];
      --j;
    }
    a[j + 1] = x;
  }
}

__device__ __forceinline__ int lower_bound(const int* a, int len, int x) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// nbr holds, per vertex v, 2*deg(v)+1 ints at offset 2*incptr[v] + v.
__global__ void __launch_bounds__(256) rows_kernel(const int* __restrict__ F, int n, const int* __restrict__ incptr,
                                                   int* __restrict__ inc_fc, int* __restrict__ nbr,
                                                   int* __restrict__ rowlen, int* __restrict__ err) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int beg = incptr[v];
  const int deg = incptr[v + 1] - beg;
  if (deg == 0) {
    atomicOr(err, kErrUnused);
    rowlen[v] = 1;
    nbr[2 * beg + v] = v;
    return;
  }
  insertion_sort(inc_fc + beg, deg);
  int* list = nbr + 2 * (long)beg + v;
  list[0] = v;
  for (int e = 0; e < deg; ++e) {
    const int fc = inc_fc[beg + e];
    const int f = fc >> 2, c = fc & 3;
    list[1 + 2 * e] = F[3 * f + (c + 1) % 3];
    list[2 + 2 * e] = F[3 * f + (c + 2) % 3];
  }
  const int len = 2 * deg + 1;
  insertion_sort(list, len);
  int u = 1;
  for (int i = 1; i < len; ++i)
    if (list[i] != list[u - 1]) list[u++] = list[i];
  if (u > 65535) atomicOr(err, kErrValence);
  rowlen[v] = u;
}

__global__ void __launch_bounds__(256) cols_kernel(const int* __restrict__ F, int n, const int* __restrict__ incptr,
                                                   const int* __restrict__ inc_fc, const int* __restrict__ nbr,
                                                   const int* __restrict__ rowptr, int* __restrict__ col,
                                                   int* __restrict__ diagpos, int2* __restrict__ inc) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int beg = incptr[v];
  const int deg = incptr[v + 1] - beg;
  const int* list = nbr + 2 * (long)beg + v;
  const int r0 = rowptr[v];
  const int len = rowptr[v + 1] - r0;
  for (int i = 0; i < len; ++i) col[r0 + i] = list[i];
  diagpos[v] = r0 + lower_bound(list, len, v);
  for (int e = 0; e < deg; ++e) {
    const int fc = inc_fc[beg + e];
    const int f = fc >> 2, c = fc & 3;
    const int nx = F[3 * f + (c + 1) % 3];
    const int pv = F[3 * f + (c + 2) % 3];
    const int sn = lower_bound(list, len, nx);
    const int sp = lower_bound(list, len, pv);
    inc[beg + e] = make_int2(fc, sn | (sp << 16));
  }
}

// Sliced-ELL: 32 x (widest row of the slice) entries per slice of 32 rows.
__global__ void __launch_bounds__(256) sell_width_kernel(const int* __restrict__ rowptr, int n,
                                                         int* __restrict__ width32) {
  const int sl = blockIdx.x * blockDim.x + threadIdx.x;
  const int nsl = (n + 31) / 32;
  if (sl >= nsl) return;
  int w = 0;
  for (int r = sl * 32; r < sl * 32 + 32 && r < n; ++r) {
    const int len = rowptr[r + 1] - rowptr[r];
    w = len > w ? len : w;
  }
  width32[sl] = 32 * w;
}

// One thread per (slice, lane): copy the row's columns, pad with the row itself (value 0 later).
// Lanes past n (last slice) are padded with the slice's first row.
__global__ void __launch_bounds__(256) sell_fill_kernel(const int* __restrict__ rowptr, const int* __restrict__ col,
                                                        int n, const int* __restrict__ sell_ptr,
                                                        int* __restrict__ sell_col) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nsl = (n + 31) / 32;
  if (t >= (long)nsl * 32) return;
  const int sl = (int)(t >> 5), lane = (int)(t & 31);
  const int r = (int)t;
  const int base = sell_ptr[sl] + lane;
  const int w = (sell_ptr[sl + 1] - sell_ptr[sl]) >> 5;
  int len = 0, r0 = 0;
  if (r < n) {
    r0 = rowptr[r];
    len = rowptr[r + 1] - r0;
  }
  const int pad = r < n ? r : sl * 32;
  for (int j = 0; j < w; ++j) sell_col[base + 32 * j] = j < len ? col[r0 + j] : pad;
}

// One warp per slice: the slice's columns as 16-bit offsets from its first row; nfar counts the
// slices with a column farther than +-32767 (a grid's neighbours are within +-(nx + 1) rows; an
// icosphere's subdivision order can put them anywhere), in which case the offsets are not used.
__global__ void __launch_bounds__(256) sell_c16_kernel(const int* __restrict__ sell_ptr,
                                                       const int* __restrict__ sell_col, int n,
                                                       short* __restrict__ c16, int* __restrict__ nfar) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nsl = (n + 31) / 32;
  const int sl = (int)(t >> 5), lane = (int)(t & 31);
  if (sl >= nsl) return;  // whole warps leave together (nsl * 32 threads are in range)
  const int b0 = sell_ptr[sl], w = (sell_ptr[sl + 1] - b0) >> 5;
  const int base = sl * 32;
  bool fits = true;
  for (int j = 0; j < w; ++j) {
    const int d = sell_col[b0 + 32 * j + lane] - base;
    fits = fits && d >= -32767 && d <= 32767;
    c16[b0 + 32 * j + lane] = (short)(fits ? d : 0);
  }
  if (!__all_sync(0xffffffffu, fits) && lane == 0) atomicAdd(nfar, 1);
}

inline int blocks_for(long work) { return (int)((work + 255) / 256); }

}  // namespace

cudaError_t launch_pattern_count(const int* F, int m, int n, int* deg, int* err, cudaStream_t st) {
  count_kernel<<<blocks_for(m), 256, 0, st>>>(F, m, n, deg, err);
  return cudaGetLastError();
}

cudaError_t launch_pattern_fill(const int* F, int m, const int* incptr, int* fill, int* inc_fc, cudaStream_t st) {
  fill_kernel<<<blocks_for(m), 256, 0, st>>>(F, m, incptr, fill, inc_fc);
  return cudaGetLastError();
}

cudaError_t launch_pattern_rows(const int* F, int n, const int* incptr, int* inc_fc, int* nbr, int* rowlen, int* err,
                                cudaStream_t st) {
  rows_kernel<<<blocks_for(n), 256, 0, st>>>(F, n, incptr, inc_fc, nbr, rowlen, err);
  return cudaGetLastError();
}

cudaError_t launch_pattern_cols(const int* F, int n, const int* incptr, const int* inc_fc, const int* nbr,
                                const int* rowptr, int* col, int* diagpos, int2* inc, int* err, cudaStream_t st) {
  (void)err;
  cols_kernel<<<blocks_for(n), 256, 0, st>>>(F, n, incptr, inc_fc, nbr, rowptr, col, diagpos, inc);
  return cudaGetLastError();
}

cudaError_t launch_sell_width(const int* rowptr, int n, int* width32, cudaStream_t st) {
  sell_width_kernel<<<blocks_for((n + 31) / 32), 256, 0, st>>>(rowptr, n, width32);
  return cudaGetLastError();
}

cudaError_t launch_sell_c16(const int* sell_ptr, const int* sell_col, int n, short* c16, int* nfar,
                            cudaStream_t st) {
  sell_c16_kernel<<<blocks_for((long)((n + 31) / 32) * 32), 256, 0, st>>>(sell_ptr, sell_col, n, c16, nfar);
  return cudaGetLastError();
}

cudaError_t launch_sell_fill(const int* rowptr, const int* col, int n, const int* sell_ptr, int* sell_col,
                             cudaStream_t st) {
  sell_fill_kernel<<<blocks_for((long)((n + 31) / 32) * 32), 256, 0, st>>>(rowptr, col, n, sell_ptr, sell_col);
  return cudaGetLastError();
}

}  // namespace ig
