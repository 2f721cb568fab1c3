// ig_device.cuh -- device helpers shared by the solver kernels: bit-level finiteness tests,
// deterministic CTA and cross-tile reductions, row loads, and the device-side loop control.
#pragma once

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
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.0;
  for (int t = threadIdx.x; t < ntiles; t += kBlock)
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __ldcg(part + t * kPartStride + i);
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

// The last CTA of an update launch decides whether the device-side loop goes on: it stops when
// every mesh of the group is done or the hard cap on iterations is reached.
__device__ __forceinline__ void loop_control(const MeshDev* __restrict__ mds, LoopCtl* ctl,
                                             cudaGraphConditionalHandle handle, int use_graph, int nmesh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->cnt, 1u);
    if (prev == gridDim.x - 1u) {
      __threadfence();
      int all = 1;
      for (int i = 0; i < nmesh; ++i) all &= (__ldcg(&mds[i].s->done) != 0);
      const int it = ctl->iter + 1;
      ctl->iter = it;
      if (all || it >= ctl->cap) {
        ctl->all_done = 1;
        if (use_graph) cudaGraphSetConditional(handle, 0u);
      }
      ctl->cnt = 0u;
    }
  }
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

// alpha_c = rz_c / (p_c . q_c) for active columns.
__device__ __noinline__ void finish_spmv(SolveScal* s, int k, const double* pq) {
  for (int c = 0; c < k; ++c) {
    if (s->active[c] == 0) {
      s->alpha[c] = 0.0;
    } else if (!positive_finite(pq[c])) {
      s->alpha[c] = 0.0;
      s->status = IG_ERR_NONFINITE;
      s->done = 1;
    } else {
      s->alpha[c] = s->rz[c] / pq[c];
    }
  }
}

// ------------------------------------------------------------------------------- finalize
template <int K>
__global__ void __launch_bounds__(kBlock) finalize_kernel(const MeshDev* __restrict__ mds,
                                                          const int2* __restrict__ tiles, IoTable io) {
  const int2 tl = tiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  double* __restrict__ out = io.out[tl.x];
#pragma unroll
  for (int rr = 0; rr < kRowsPerThread; ++rr) {
    const long row = (long)tl.y * kTileRows + rr * kBlock + threadIdx.x;
    if (row < md.n) {
#pragma unroll
      for (int c = 0; c < K; ++c) out[row * K + c] = md.x[row * K + c];
    }
  }
}

}  // namespace
}  // namespace ig
