// ig_device.cuh -- device helpers shared by the solver kernels: bit-level finiteness tests,
// deterministic CTA and cross-tile reductions, row loads, and the device-side loop control.
#pragma once

#include "ig_f32.cuh"
#include "ig_internal.cuh"

namespace ig {
namespace {

template <int K>
struct KP {
  static constexpr int v = (K == 3) ? 4 : K;
};

__device__ __forceinline__ bool positive_finite(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && (b & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool is_finite(double x) {
  return (__double_as_longlong(x) & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}

// Thread j of the CTA adds the partials of tiles j, j + kBlock, j + 2 kBlock, ... in that order
// (the association is fixed by the tile count alone, so the result is deterministic). Loads go in
// batches of 4 tiles so that a thread has several L2 requests in flight.
template <int NV>
__device__ __noinline__ void gather_partials_impl(const double* __restrict__ part, int ntiles, double* out) {
  double v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.0;
  for (int t = threadIdx.x; t < ntiles; t += 4 * kBlock) {
    // four tiles' loads in flight together; a tile past the end reads as +0, which leaves the
    // sum unchanged
    double b[4][NV];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int tu = t + u * kBlock;
#pragma unroll
      for (int i = 0; i < NV; ++i) b[u][i] = tu < ntiles ? __ldcg(part + tu * kPartStride + i) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < NV; ++i) v[i] += b[u][i];
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) out[i] = v[i];
}

// (kept out of line: only the last CTA of a reduction runs it)
template <int NV>
__device__ __forceinline__ void gather_partials(const double* __restrict__ part, int ntiles, double (&v)[NV]) {
  gather_partials_impl<NV>(part, ntiles, v);
}

// Sum v[0..NV) over the CTA; thread 0 receives the totals. sh holds NV*kBlock doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
#pragma unroll
  for (int i = 0; i < NV; ++i) sh[i * kBlock + threadIdx.x] = v[i];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double a = sh[i * kBlock + threadIdx.x];
#pragma unroll
      for (int w = 1; w < kBlock / 32; ++w) a += sh[i * kBlock + threadIdx.x + 32 * w];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      v[i] = a;
    }
  }
  __syncthreads();
}

// Block-sum v, publish the tile's partials, and return true in the last CTA of the mesh, whose
// thread 0 then holds the mesh totals (partials added in tile order, so the result does not
// depend on which CTA finished last).
template <int NV>
__device__ __forceinline__ bool reduce_tiles(double (&v)[NV], double* part, int tile, int ntiles, unsigned int* cnt,
                                             double* sh) {
  __shared__ int s_last;
  block_sum<NV>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) part[tile * kPartStride + i] = v[i];
    __threadfence();
    const unsigned prev = atomicAdd(cnt, 1u);
    s_last = (prev == (unsigned)ntiles - 1u);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  gather_partials<NV>(part, ntiles, v);
  block_sum<NV>(v, sh);
  if (threadIdx.x == 0) *cnt = 0u;
  return true;
}

template <int K>
__device__ __forceinline__ void load_row(const double* __restrict__ p, long row, double (&v)[K]) {
  if constexpr (K == 3 || K == 4) {
    const double2* q = reinterpret_cast<const double2*>(p + row * KP<K>::v);
    const double2 a = q[0], b = q[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x;
    if constexpr (K == 4) v[3] = b.y;
  } else if constexpr (K == 2) {
    const double2 a = reinterpret_cast<const double2*>(p + row * 2)[0];
    v[0] = a.x; v[1] = a.y;
  } else {
    v[0] = p[row];
  }
}

// Row store into a padded [n][KP] vector (16-byte stores where the row allows).
template <int K>
__device__ __forceinline__ void store_row(double* __restrict__ p, long row, const double (&v)[K]) {
  if constexpr (K == 3 || K == 4) {
    double2* q = reinterpret_cast<double2*>(p + row * KP<K>::v);
    q[0] = make_double2(v[0], v[1]);
    if constexpr (K == 4) q[1] = make_double2(v[2], v[3]);
    else p[row * 4 + 2] = v[2];
  } else if constexpr (K == 2) {
    reinterpret_cast<double2*>(p + row * 2)[0] = make_double2(v[0], v[1]);
  } else {
    p[row] = v[0];
  }
}

template <int K>
__device__ __forceinline__ void load_row32(const float* __restrict__ p, long row, float (&v)[K]);

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// A stored value in the arithmetic type: a float value of the FP32 operator is taken into FP64
// exactly, with integer instructions (the FP64 residual of the FP32-geometry mode).
template <typename TX, typename TA>
__device__ __forceinline__ TX to_arith(TA a) {
  if constexpr (sizeof(TX) == 8 && sizeof(TA) == 4) return f32_to_f64(a);
  else return (TX)a;
}

// acc[c] = sum over the stored entries of row `row` of A[e] * X(col_e, c), where X is read by
// the gather functor (x(col, v) fills v[0..K)). Uses the sliced-ELL layout when the mesh has one
// (a warp's rows share one slice, so the loop count is uniform and each slot is one contiguous
// load for the warp) and plain CSR otherwise.
template <int K, typename TA, typename TX, typename G>
__device__ __forceinline__ void row_product(const MeshDev& md, const TA* __restrict__ A, long row, const G& gather,
                                            TX (&acc)[K]) {
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = TX(0);
  if (md.sell_ptr) {
    const int sl = (int)(row >> 5);
    int b0, w;
    if (md.sell_w) {  // slices of one width: the offset is computed, not loaded
      w = md.sell_w;
      b0 = sl * 32 * w;
    } else {
      b0 = __ldg(md.sell_ptr + sl);
      w = (__ldg(md.sell_ptr + sl + 1) - b0) >> 5;
    }
    const int base = b0 + (int)(row & 31);
    const int* __restrict__ sc = md.sell_col;
    if constexpr (sizeof(TX) == 4) {
      // FP32: up to 8 slots at once (a mesh row has ~7): all column/value loads, then the gathers.
      // A mesh whose columns all fit reads them as 16-bit offsets from the slice's first row.
      const bool c16 = md.sell_c16 != nullptr;
      const short* __restrict__ s16 = md.sell_c16;
      const int rbase = sl << 5;
      for (int j0 = 0; j0 < w; j0 += 8) {
        int cj[8];
        TA aj[8];
        if (c16) {
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (j0 + u < w) {
              cj[u] = rbase + (int)__ldg(s16 + base + 32 * (j0 + u));
              aj[u] = __ldg(A + base + 32 * (j0 + u));
            }
        } else {
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (j0 + u < w) {
              cj[u] = __ldg(sc + base + 32 * (j0 + u));
              aj[u] = __ldg(A + base + 32 * (j0 + u));
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (j0 + u < w) {
            TX v[K];
            gather(IG_IN_RANGE(cj[u], md.n, md.err) ? cj[u] : 0, v);
#pragma unroll
            for (int c = 0; c < K; ++c) acc[c] = fma_t((TX)aj[u], v[c], acc[c]);
          }
      }
    } else {
#pragma unroll 4
      for (int j = 0; j < w; ++j) {
        const int e = base + 32 * j;
        const TX a = to_arith<TX>(__ldg(A + e));
        TX v[K];
        const int cj = __ldg(sc + e);
        gather(IG_IN_RANGE(cj, md.n, md.err) ? cj : 0, v);
#pragma unroll
        for (int c = 0; c < K; ++c) acc[c] = fma_t(a, v[c], acc[c]);
      }
    }
  } else {
    const int e0 = __ldg(md.rowptr + row), e1 = __ldg(md.rowptr + row + 1);
    for (int e = e0; e < e1; ++e) {
      const TX a = to_arith<TX>(__ldg(A + e));
      TX v[K];
      const int cj = __ldg(md.col + e);
      gather(IG_IN_RANGE(cj, md.n, md.err) ? cj : 0, v);
#pragma unroll
      for (int c = 0; c < K; ++c) acc[c] = fma_t(a, v[c], acc[c]);
    }
  }
}

// Gathers: rows of the padded p vectors, columns of an [K][n] vector, rows of an [n][K] vector.
template <int K>
struct GatherP64 {
  const double* p;
  __device__ __forceinline__ void operator()(int j, double (&v)[K]) const { load_row<K>(p, j, v); }
};
template <int K>
struct GatherP32 {
  const float* p;
  __device__ __forceinline__ void operator()(int j, float (&v)[K]) const { load_row32<K>(p, j, v); }
};
template <int K>
struct GatherSoA64 {
  const double* x;
  long n;
  __device__ __forceinline__ void operator()(int j, double (&v)[K]) const {
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = x[c * n + j];
  }
};
template <int K>
struct GatherAoS64 {
  const double* x;
  __device__ __forceinline__ void operator()(int j, double (&v)[K]) const {
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = x[(long)j * K + c];
  }
};

// ------------------------------------------------------------------------------- warp and tile sums
// Transposed warp sum. In a plain butterfly every lane adds every value at each of the five
// levels; here, at the first levels, a lane keeps half of its values and sends the other half to
// its partner, so NV <= 8 values cost 9 shuffles and 9 adds per lane (NV <= 4: 6 and 6) instead of
// 5 NV of each. Afterwards lane L holds the warp total of value warp_sum_index<NV>(L), and the
// lanes selected by warp_sum_writer<NV>(L) hold each total once. The additions are in a fixed
// order, so the sums are deterministic. (FP64 adds are scarce on this GPU: 2 per clock per SM.)
template <int NV>
__device__ __forceinline__ int warp_sum_index(int lane) {
  if constexpr (NV <= 2) return 0;
  else if constexpr (NV <= 4) return ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
  else return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}
template <int NV>
__device__ __forceinline__ bool warp_sum_writer(int lane) {
  if constexpr (NV <= 2) return lane == 0;
  else if constexpr (NV <= 4) return (lane & 0x13) == 0;
  else return (lane & 3) == 0;
}

template <int NV, typename T>
__device__ __forceinline__ T warp_sum_transposed(T (&v)[NV], int lane) {
  static_assert(NV >= 1 && NV <= 8, "at most 8 values");
  if constexpr (NV <= 2) {
    // plain butterfly on the (one or two) values; lane 0 returns value 0 and v[] holds both totals
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    return v[0];
  } else if constexpr (NV <= 4) {
    T a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = i < NV ? v[i] : T(0);
    const bool h8 = (lane & 8) != 0, h4 = (lane & 4) != 0;
    T b[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const T keep = h8 ? a[2 + i] : a[i];
      const T send = h8 ? a[i] : a[2 + i];
      b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    T c;
    {
      const T keep = h4 ? b[1] : b[0];
      const T send = h4 ? b[0] : b[1];
      c = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    c += __shfl_xor_sync(0xffffffffu, c, 16);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
  } else {
    T a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = i < NV ? v[i] : T(0);
    const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0, h4 = (lane & 4) != 0;
    T b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const T keep = h16 ? a[4 + i] : a[i];
      const T send = h16 ? a[i] : a[4 + i];
      b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    T c[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const T keep = h8 ? b[2 + i] : b[i];
      const T send = h8 ? b[i] : b[2 + i];
      c[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    T d;
    {
      const T keep = h4 ? c[1] : c[0];
      const T send = h4 ? c[0] : c[1];
      d = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    d += __shfl_xor_sync(0xffffffffu, d, 2);
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    return d;
  }
}

constexpr int kWarps = kBlock / 32;

// Sum the per-thread values v[0..NV) over the CTA: each warp adds its lanes (in T: FP32 for the
// mixed-precision kernels, FP64 otherwise), then threads 0..NV-1 add the kWarps warp totals in FP64
// in warp order and write them to out[0..NV). red holds NV * kWarps doubles; a caller that sums
// consecutive tiles alternates between two such buffers, so that one barrier per tile suffices
// (a warp can reach the buffer again only after the next tile's barrier, which the readers of
// this tile pass after their reads).
template <int NV, typename T>
__device__ __forceinline__ void tile_reduce(T (&v)[NV], double* red, double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T w = warp_sum_transposed<NV>(v, lane);
  if constexpr (NV <= 2) {
    if (lane == 0)
#pragma unroll
      for (int i = 0; i < NV; ++i) red[i * kWarps + warp] = (double)v[i];
  } else {
    const int idx = warp_sum_index<NV>(lane);
    if (warp_sum_writer<NV>(lane) && idx < NV) red[idx * kWarps + warp] = (double)w;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double a = red[threadIdx.x * kWarps];
#pragma unroll
    for (int j = 1; j < kWarps; ++j) a += red[threadIdx.x * kWarps + j];
    out[threadIdx.x] = a;
  }
}

// ------------------------------------------------------------------------------- persistent tiles
// The tilings of a mesh: 0 the FP64 solver's, 1 the mixed-precision SpMV's and p-update's, 2 the
// mixed-precision update's (one wave of large tiles on meshes of at least kBigRows rows, the
// tiling 1 otherwise, so that the chunked lists of smaller meshes serve both).
__device__ __forceinline__ int tile_count(const MeshDev& md, int tiling) {
  return tiling == 0 ? md.ntiles : (tiling == 1 ? md.ntiles32 : md.ntiles32u);
}

// Per-CTA view of the mesh whose tiles the CTA is working on: a copy of its MeshDev and of the
// scalars the kernels read, taken once per mesh switch. Every CTA of a launch reads the same few
// scalars; reading them through one thread per CTA keeps them off a single hot L2 line, and the
// copy in shared memory keeps the mesh's pointers out of the way of the kernels' global stores.
struct ScalSnap {
  double alpha[kMaxK];
  double beta[kMaxK];
  double scale[kMaxK];
  int act64[kMaxK];
  int done;
  int phase;
};

struct TileCtx {
  MeshDev md;
  ScalSnap sn;
  double red[2][8 * kWarps];  // tile sums, double-buffered
  double tot[8];              // mesh totals in the CTA that completes a mesh
  SolveScal cur;              // the mesh's scalars as the CTA that completes it found them
  int last;
};

__device__ __forceinline__ void load_mesh(const MeshDev* __restrict__ mds, int i, TileCtx& tc) {
  __syncthreads();  // every thread is done with the previous mesh's view
  static_assert(sizeof(MeshDev) % 4 == 0, "MeshDev is copied as 4-byte words");
  const unsigned* src = reinterpret_cast<const unsigned*>(mds + i);
  unsigned* dst = reinterpret_cast<unsigned*>(&tc.md);
  for (int j = threadIdx.x; j < (int)(sizeof(MeshDev) / 4); j += kBlock) dst[j] = __ldg(src + j);
  if (threadIdx.x == 0) {
    const SolveScal* s = mds[i].s;
    tc.sn.done = s->done;
    tc.sn.phase = s->phase;
#pragma unroll
    for (int c = 0; c < kMaxK; ++c) {
      tc.sn.alpha[c] = s->alpha[c];
      tc.sn.beta[c] = s->beta[c];
      tc.sn.scale[c] = s->scale[c];
      tc.sn.act64[c] = s->active64[c];
    }
  }
  __syncthreads();
}

// The loop kernels run one CTA per resident slot; CTA b takes the flat tiles b, b + G, b + 2G, ...
// (G = gridDim.x). A tile's sums go to the mesh's part[tile]; each CTA counts the tiles it did
// per run of consecutive tiles of one mesh and adds that count to the mesh's counter with one
// atomic. The CTA whose addition completes the mesh adds the partials in tile order
// (deterministic, independent of G and of any batch) and calls finish(md, scalars, totals) on
// warp 0, with a shared-memory copy of the mesh's scalars to read (writes go to md.s).
template <int NV, typename Finish>
__device__ __forceinline__ void flush_tiles(TileCtx& tc, int tiling, unsigned run, int cnt_idx,
                                            const Finish& finish) {
  const int ntiles = tile_count(tc.md, tiling);
  unsigned int* cnt = &tc.md.s->cnt[cnt_idx];
  if (threadIdx.x < NV) __threadfence();  // the tile sums this thread wrote, before the count
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(cnt, run);
    tc.last = (prev + run == (unsigned)ntiles);
  }
  __syncthreads();
  if (tc.last) {
    __threadfence();
    // the mesh's scalars are read into shared memory while the partials are gathered, so that
    // the finish step does not wait on one global load after another
    static_assert(sizeof(SolveScal) % 4 == 0 && sizeof(SolveScal) / 4 <= kBlock, "SolveScal copy");
    if (threadIdx.x < (int)(sizeof(SolveScal) / 4))
      reinterpret_cast<unsigned*>(&tc.cur)[threadIdx.x] =
          __ldcg(reinterpret_cast<const unsigned*>(tc.md.s) + threadIdx.x);
    double v[NV];
    gather_partials<NV>(tc.md.part, ntiles, v);
    tile_reduce<NV>(v, tc.red[0], tc.tot);
    __syncthreads();
    if (threadIdx.x < 32) {
      if (threadIdx.x == 0) *cnt = 0u;
      finish(tc.md, tc.cur, tc.tot);
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------- active list
// Exclusive scan of three counters over the CTA (thread order), with the CTA totals.
__device__ __forceinline__ void block_exscan3(int a, int b, int c, int& ea, int& eb, int& ec, int& ta, int& tb,
                                              int& tc) {
  __shared__ int ws[3][kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int ia = a, ib = b, ic = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int xa = __shfl_up_sync(0xffffffffu, ia, o);
    const int xb = __shfl_up_sync(0xffffffffu, ib, o);
    const int xc = __shfl_up_sync(0xffffffffu, ic, o);
    if (lane >= o) {
      ia += xa;
      ib += xb;
      ic += xc;
    }
  }
  if (lane == 31) {
    ws[0][warp] = ia;
    ws[1][warp] = ib;
    ws[2][warp] = ic;
  }
  __syncthreads();
  int pa = 0, pb = 0, pc = 0;
  ta = tb = tc = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    if (w < warp) {
      pa += ws[0][w];
      pb += ws[1][w];
      pc += ws[2][w];
    }
    ta += ws[0][w];
    tb += ws[1][w];
    tc += ws[2][w];
  }
  ea = pa + ia - a;
  eb = pb + ib - b;
  ec = pc + ic - c;
  __syncthreads();
}

// Start table of one grid: entry g = (list position j, local tile, mesh, tile count) of the chunk
// [g·chunk, (g+1)·chunk) of the listed tiles, or a zero count past them. off[0..ns] are the tile
// offsets of the listed meshes (off[ns] = total).
__device__ __forceinline__ void fill_starts(int4* st, int grid, int chunk, int total, const int* off,
                                            const int* mesh, int ns) {
  for (int g = threadIdx.x; g < grid; g += kBlock) {
    const long x = (long)g * chunk;
    if (x >= total || ns == 0) {
      st[g] = make_int4(0, 0, -1, 0);
      continue;
    }
    int lo = 0, hi = ns - 1;  // the largest j with off[j] <= x
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= x) lo = mid;
      else hi = mid - 1;
    }
    const int cnt = total - x < chunk ? (int)(total - x) : chunk;
    st[g] = make_int4(lo, (int)(x - off[lo]), mesh[lo], cnt);
  }
}

// Build one list (run by every thread of one CTA, after every other CTA of the launch is done
// with it): the meshes that are not done and satisfy sel(s). Big meshes go to `big`; the others to
// `mesh` with their tile offsets (FP64 tiling in off64 when given, mixed tiling in off32) and the
// start tables: CTA g of a loop kernel takes the listed tiles [g·chunk, (g+1)·chunk).
template <typename Sel>
__device__ __forceinline__ void build_list(const MeshDev* __restrict__ mds, int nmesh, const Sel& sel, int* mesh,
                                           int* off64, int* off32, int4* st64, int g64, int4* st32, int g32,
                                           int* big, int& ns, int& nbig, int& ndone) {
  int tot64 = 0, tot32 = 0;
  ns = nbig = ndone = 0;
  for (int i0 = 0; i0 < nmesh; i0 += kBlock) {
    const int i = i0 + threadIdx.x;
    int small = 0, isbig = 0, dn = 0, c64 = 0, c32 = 0;
    if (i < nmesh) {
      const SolveScal* s = mds[i].s;
      dn = __ldcg(&s->done) != 0;
      if (!dn && sel(s)) {
        if (mds[i].n >= kBigRows) {
          isbig = 1;
        } else {
          small = 1;
          c64 = mds[i].ntiles;
          c32 = mds[i].ntiles32;
        }
      }
    }
    int e0, e1, e2, t0, t1, t2;
    block_exscan3(small, c64, c32, e0, e1, e2, t0, t1, t2);
    if (small) {
      mesh[ns + e0] = i;
      if (off64) off64[ns + e0] = tot64 + e1;
      off32[ns + e0] = tot32 + e2;
    }
    int f0, f1, f2, u0, u1, u2;
    block_exscan3(isbig, dn, 0, f0, f1, f2, u0, u1, u2);
    if (isbig) big[nbig + f0] = i;
    ns += t0;
    tot64 += t1;
    tot32 += t2;
    nbig += u0;
    ndone += u1;
  }
  const int ch64 = tot64 > 0 && g64 > 0 ? (tot64 + g64 - 1) / g64 : 1;
  const int ch32 = tot32 > 0 && g32 > 0 ? (tot32 + g32 - 1) / g32 : 1;
  if (threadIdx.x == 0) {
    if (off64) off64[ns] = tot64;
    off32[ns] = tot32;
  }
  __syncthreads();  // the offsets above are visible to the whole CTA
  // each CTA's start: the listed mesh whose tiles contain the chunk's first tile (binary search
  // over the offsets, one CTA entry per thread)
  if (st64) fill_starts(st64, g64, ch64, tot64, off64, mesh, ns);
  fill_starts(st32, g32, ch32, tot32, off32, mesh, ns);
}

struct SelAll {
  __device__ bool operator()(const SolveScal*) const { return true; }
};
struct SelApply {
  __device__ bool operator()(const SolveScal* s) const { return __ldcg(&s->phase) == kPhaseApply; }
};

// The active list: every mesh that is not done.
__device__ __noinline__ void rebuild_active(const MeshDev* __restrict__ mds, LoopCtl* ctl) {
  int ns, nbig, ndone;
  build_list(mds, ctl->nmesh, SelAll{}, ctl->act_mesh, ctl->act_off64, ctl->act_off32, ctl->start64, ctl->grid64,
             ctl->start32, ctl->grid32, ctl->big_mesh, ns, nbig, ndone);
  if (threadIdx.x == 0) {
    ctl->nact = ns;
    ctl->nbig = nbig;
    ctl->ndone_list = ndone;
  }
}

// The Apply list (mixed precision, mixed tiling): meshes not done and in the Apply phase.
__device__ __noinline__ void rebuild_apply(const MeshDev* __restrict__ mds, LoopCtl* ctl) {
  int ns, nbig, ndone;
  build_list(mds, ctl->nmesh, SelApply{}, ctl->app_mesh, nullptr, ctl->app_off32, nullptr, 0, ctl->app_start32,
             ctl->grid32, ctl->app_big, ns, nbig, ndone);
  if (threadIdx.x == 0) ctl->napp_big = nbig;
}

// The tiles one CTA of a loop kernel takes: tiles b, b + G, ... of every big mesh (b =
// blockIdx.x, G = gridDim.x), then its chunk of the chunked list. One walker for both parts, so
// that a kernel's tile body is compiled once.
struct TileWalk {
  int nbig, bi, mi, lt, j, left;  // bi < nbig: in the big list; then the chunk (left tiles to go)
  __device__ __forceinline__ void chunk(const ListRef& L) {
    const int4 st = L.start[blockIdx.x];
    bi = nbig;
    j = st.x;
    lt = st.y;
    mi = st.z;
    left = st.w;
  }
  __device__ __forceinline__ void begin(const ListRef& L) {
    nbig = *L.nbig;
    bi = 0;
    left = 0;
    j = 0;
    if (nbig > 0) {
      mi = L.big[0];
      lt = blockIdx.x;
    } else {
      chunk(L);
    }
  }
  __device__ __forceinline__ bool more() const { return bi < nbig || left > 0; }
  // after the mesh mi is loaded (nt tiles): false when the current big mesh has no more tiles for
  // this CTA (the walker then moved on; call more() again)
  __device__ __forceinline__ bool here(const ListRef& L, int nt) {
    if (bi < nbig && lt >= nt) {
      if (++bi < nbig) {
        mi = L.big[bi];
        lt = blockIdx.x;
      } else {
        chunk(L);
      }
      return false;
    }
    return true;
  }
  __device__ __forceinline__ void next(const ListRef& L, int nt) {
    if (bi < nbig) {
      lt += gridDim.x;
    } else {
      --left;
      if (++lt == nt) {
        ++j;
        lt = 0;
        if (left > 0) mi = L.act[j];
      }
    }
  }
};

// body(md, tile, red, out) does the tile's work and sums its NV values into out with
// tile_reduce(v, red, out); active(sn) says whether a mesh takes part in this launch (uniform per
// CTA). tiling: see tile_count; cnt_idx selects the mesh counter.
template <int NV, typename Active, typename Body, typename Finish>
__device__ __forceinline__ void tile_loop(const MeshDev* __restrict__ mds, const ListRef& L, int tiling, int cnt_idx,
                                          TileCtx& tc, const Active& active, const Body& body,
                                          const Finish& finish) {
  TileWalk w;
  w.begin(L);
  int cur = -1, buf = 0;
  unsigned run = 0;
  while (w.more()) {
    if (w.mi != cur) {
      if (run) flush_tiles<NV>(tc, tiling, run, cnt_idx, finish);
      cur = w.mi;
      run = 0;
      load_mesh(mds, cur, tc);
    }
    const int nt = tile_count(tc.md, tiling);
    if (!w.here(L, nt)) continue;
    if (active(tc.sn)) {
      body(tc.md, w.lt, tc.red[buf], tc.md.part + (long)w.lt * kPartStride);
      buf ^= 1;
      ++run;
    }
    w.next(L, nt);
  }
  if (run) flush_tiles<NV>(tc, tiling, run, cnt_idx, finish);
}

// Tile loop without sums.
template <typename Active, typename Body>
__device__ __forceinline__ void tile_loop_plain(const MeshDev* __restrict__ mds, const ListRef& L, int tiling,
                                                TileCtx& tc, const Active& active, const Body& body) {
  TileWalk w;
  w.begin(L);
  int cur = -1;
  while (w.more()) {
    if (w.mi != cur) {
      cur = w.mi;
      load_mesh(mds, cur, tc);
    }
    const int nt = tile_count(tc.md, tiling);
    if (!w.here(L, nt)) continue;
    if (active(tc.sn)) body(tc.md, w.lt);
    w.next(L, nt);
  }
}

// The last CTA of an update launch decides whether the device-side loop goes on: it stops when
// every mesh of the group is done, the hard cap on iterations is reached, or (serving) a member
// that was running has finished. It rebuilds the active list when more meshes are done.
__device__ __forceinline__ void loop_control(const MeshDev* __restrict__ mds, LoopCtl* ctl,
                                             cudaGraphConditionalHandle handle, int use_graph) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->cnt, 1u);
    s_last = (prev == gridDim.x - 1u);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int nmesh = ctl->nmesh;
  int ndone = 0, apply = 0;
  for (int i0 = 0; i0 < nmesh; i0 += kBlock) {
    const int i = i0 + threadIdx.x;
    int d = 0, ap = 0;
    if (i < nmesh) {
      const SolveScal* s = mds[i].s;
      d = __ldcg(&s->done) != 0;
      ap = !d && __ldcg(&s->phase) == kPhaseApply;
    }
    ndone += __syncthreads_count(d);
    apply |= __syncthreads_or(ap);
  }
  const int rebuild = ndone > ctl->ndone_list && ndone < nmesh;
  __syncthreads();
  if (rebuild) rebuild_active(mds, ctl);
  if (apply && ctl->app_mesh) rebuild_apply(mds, ctl);
  if (threadIdx.x == 0) {
    ctl->any_apply = apply;
    const int it = ctl->iter + 1;
    ctl->iter = it;
    if (ndone == nmesh || it >= ctl->cap || ndone > ctl->ndone_start) {
      ctl->all_done = 1;
      if (use_graph) cudaGraphSetConditional(handle, 0u);
    }
    ctl->cnt = 0u;
  }
}

// Loop control of a group of one mesh (the FP64 and the mixed-precision update), on lane 0 of the
// CTA that completes the mesh, right after its finish step: the loop stops when the mesh is done
// or the cap is reached. The iteration
// counter and the cap were read at the kernel's entry (only this step writes the counter), and
// done is the finish step's own result, so the step makes no global read. A launch in which the
// mesh takes no part is stopped by its CTA 0 at entry, so every launch either completes the mesh
// (and counts towards the cap) or stops the loop. (A group of several meshes needs every CTA of
// the launch to have finished, for the list rebuilds: loop_control.)
__device__ __forceinline__ void single_loop_control(int done, int iter, int cap, LoopCtl* ctl,
                                                    cudaGraphConditionalHandle handle, int use_graph) {
  const int it = iter + 1;
  ctl->iter = it;
  if (done || it >= cap) {
    ctl->all_done = 1;
    if (use_graph) cudaGraphSetConditional(handle, 0u);
  }
}

// Start of a solve or of a serving round: list every mesh that is not done.
__global__ void __launch_bounds__(kBlock) list_kernel(const MeshDev* __restrict__ mds, LoopCtl* ctl) {
  rebuild_active(mds, ctl);
}

// Row loads of [n][KP] float vectors (KP = 4 when K = 3: one aligned 16-byte load).
template <int K>
__device__ __forceinline__ void load_row32(const float* __restrict__ p, long row, float (&v)[K]) {
  if constexpr (K == 3 || K == 4) {
    const float4 a = reinterpret_cast<const float4*>(p + row * 4)[0];
    v[0] = a.x; v[1] = a.y; v[2] = a.z;
    if constexpr (K == 4) v[3] = a.w;
  } else if constexpr (K == 2) {
    const float2 a = reinterpret_cast<const float2*>(p + row * 2)[0];
    v[0] = a.x; v[1] = a.y;
  } else {
    v[0] = p[row];
  }
}

// alpha_c = rz_c / (p_c . q_c) for active columns. The finish steps run on the 32 lanes of warp 0
// of the CTA that completes a mesh: lane c handles column c (its divisions and square roots
// run side by side instead of one after another on one thread), lane 0 the mesh's own fields.
// They read the scalars from cur (a copy in shared memory) and write them to s.
__device__ __noinline__ void finish_spmv(SolveScal* s, const SolveScal& cur, int k, const double* pq) {
  const int c = threadIdx.x & 31;
  int bad = 0;
  if (c < k) {
    if (cur.active[c] == 0) {
      s->alpha[c] = 0.0;
    } else if (!positive_finite(pq[c])) {
      s->alpha[c] = 0.0;
      bad = 1;
    } else {
      s->alpha[c] = cur.rz[c] / pq[c];
    }
  }
  if (__any_sync(0xffffffffu, bad) && c == 0) {
    s->status = IG_ERR_NONFINITE;
    s->done = 1;
  }
}

// ------------------------------------------------------------------------------- finalize
template <int K>
__global__ void __launch_bounds__(kBlock) finalize_kernel(const MeshDev* __restrict__ mds,
                                                          const int2* __restrict__ tiles, IoTable io) {
  const int2 tl = tiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const long nn = md.n;
  const long t0 = (long)tl.y * md.tile_rows;
  const long t1 = t0 + md.tile_rows < nn ? t0 + md.tile_rows : nn;
  double* __restrict__ out = io.out[tl.x];
  for (long row = t0 + threadIdx.x; row < t1; row += kBlock) {
#pragma unroll
    for (int c = 0; c < K; ++c) out[row * K + c] = md.x[c * nn + row];
  }
}

}  // namespace
}  // namespace ig
