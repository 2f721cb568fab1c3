// ig_pcg_mixed.cu -- mixed-precision solve of A X = RHS (forward and adjoint systems of §7.1 /
// §5.2) to an FP64 relative residual: FP32 Jacobi-PCG on the FP32 copy of A inside an FP64
// iterative refinement whose residuals use the FP64 operator.
//
//   x64 = 0, r64 = rhs
//   repeat:  r32 = r64 / ||r64||            (per column; unit-norm inner right-hand side)
//            solve A32 d = r32 by FP32 Jacobi-PCG to inner_tol (dot products summed in FP64)
//            x64 += ||r64|| d
//            r64 = rhs - A64 x64 in FP64; stop when ||r64|| / ||rhs|| <= rel_tol
//
// It runs inside the same three-kernel iteration as the FP64 solver, with a per-mesh phase:
//   Inner   : spmv q32 = A32 p32 | update x32, r32, (r.z, r.r) | pupdate p32
//   Apply   : set by update when the inner solve converged; pupdate adds ||r64|| d into x64
//   (next)  : spmv computes r64 = rhs - A64 x64 and its norms (the refinement residual)
//   Restart : update forms r32 = r64 / ||r64||, d = 0; pupdate sets p32 = z32
// so a refinement costs one iteration slot whose SpMV runs in FP64, and no extra launches.
// FP64 arithmetic is used only for the residual SpMV, the x64 update and the reductions.
#include "ig_device.cuh"

namespace ig {

namespace {

template <int K>
struct KPm {
  static constexpr int v = (K == 3) ? 4 : K;
};

// The mixed-precision kernels take a tile in passes of kTileRows rows (kRowsPerThread per thread);
// a thread adds its rows' FP32 products across the passes of a tile (at most 64 passes, 256
// terms), the warps add their lanes in FP32 and the tile's warps and tiles are added in FP64.
template <int NV>
struct PassSum {
  float s[NV];
  __device__ __forceinline__ PassSum() {
#pragma unroll
    for (int i = 0; i < NV; ++i) s[i] = 0.f;
  }
  __device__ __forceinline__ void add(const float (&x)[NV]) {
#pragma unroll
    for (int i = 0; i < NV; ++i) s[i] += x[i];
  }
};

// ------------------------------------------------------------------------------- bookkeeping
__device__ __noinline__ void finish_init_mixed(SolveScal* s, int k, const double* acc, double tol, double inner_tol,
                                               int max_iter, int max_refine) {
  int nact = 0, bad = 0;
  for (int c = 0; c < kMaxK; ++c) {
    const double bb = c < k ? acc[c] : 0.0;
    if (c < k && !is_finite(bb)) bad = 1;
    const int act = (c < k && positive_finite(bb)) ? 1 : 0;
    s->rhs2[c] = bb;
    s->bnorm2[c] = 0.0;
    s->active64[c] = act;
    s->active[c] = 0;
    s->relres[c] = act ? 1.0 : 0.0;
    s->relres_inner[c] = 0.0;
    s->scale[c] = act ? sqrt(bb) : 1.0;
    s->rz[c] = 0.0;
    s->alpha[c] = 0.0;
    s->beta[c] = 0.0;
    s->trueres[c] = -1.0;
    nact += act;
  }
  s->k = k;
  s->cnt[0] = 0u;
  s->cnt[1] = 0u;
  s->iter = 0;
  s->refine = 0;
  s->inner_iter = 0;
  s->inner_cap = max_iter < 4000 ? max_iter : 4000;
  s->phase = kPhaseRestart;
  s->tol = tol;
  s->inner_tol = inner_tol;
  s->max_iter = max_iter;
  s->max_refine = max_refine;
  s->status = bad ? IG_ERR_NONFINITE : IG_OK;
  s->done = (bad || nact == 0) ? 1 : 0;
}

// The finish steps below run on the 32 lanes of warp 0 of the CTA that completes a mesh: lane c
// handles column c, lane 0 the mesh's own fields (written after the warp's votes). They read the
// scalars from cur, a shared-memory copy, and write them to s.

// After r64 = rhs - A64 x64: FP64 convergence test per column, the scale of the next inner
// right-hand side, and the refinement cap.
__device__ __noinline__ void finish_residual(SolveScal* s, const SolveScal& cur, int k, const double* res2) {
  const int c = threadIdx.x & 31;
  const int refine = cur.refine + 1;
  int act = 0, bad = 0;
  if (c < k && cur.active64[c] != 0) {
    if (!is_finite(res2[c])) {
      bad = 1;
    } else {
      const double rel = sqrt(res2[c] / cur.rhs2[c]);
      s->relres[c] = rel;
      if (rel <= cur.tol || !positive_finite(res2[c])) {
        s->active64[c] = 0;
      } else {
        s->scale[c] = sqrt(res2[c]);
        act = 1;
      }
    }
  }
  const int nact = __popc(__ballot_sync(0xffffffffu, act));
  const int anybad = __any_sync(0xffffffffu, bad);
  if (c == 0) {
    s->refine = refine;
    if (anybad) {
      s->status = IG_ERR_NONFINITE;
      s->done = 1;
    } else if (nact == 0) {
      s->done = 1;
    } else if (refine >= cur.max_refine || cur.iter >= cur.max_iter) {
      s->status = IG_ERR_NOT_CONVERGED;
      s->done = 1;
    } else {
      s->phase = kPhaseRestart;
    }
  }
}

// After forming r32 = r64 / scale: start a new inner solve. Returns (on lane 0) the new phase.
__device__ __noinline__ int finish_restart(SolveScal* s, const SolveScal& cur, int k, const double* acc) {
  const int c = threadIdx.x & 31;
  int act = 0;
  if (c < k) {
    act = (cur.active64[c] && positive_finite(acc[k + c])) ? 1 : 0;
    s->active[c] = act;
    s->rz[c] = acc[c];
    s->bnorm2[c] = acc[k + c];
    s->alpha[c] = 0.0;
    s->beta[c] = 0.0;
    s->relres_inner[c] = act ? 1.0 : 0.0;
  }
  const int nact = __popc(__ballot_sync(0xffffffffu, act));
  const int phase = nact ? kPhaseInner : kPhaseApply;
  if (c == 0) {
    s->inner_iter = 0;
    s->phase = phase;
  }
  return phase;
}

// Inner FP32 iteration: inner convergence test, beta, switch to Apply when the inner solve is done.
// Returns (on lane 0) the phase after it, or -1 when the mesh is done (a non-finite sum).
__device__ __noinline__ int finish_update_mixed(SolveScal* s, const SolveScal& cur, int k, const double* acc) {
  const int c = threadIdx.x & 31;
  int act = 0, bad = 0;
  if (c < k && cur.active[c] != 0) {
    const double rzn = acc[c], rr = acc[k + c];
    if (!is_finite(rzn) || !is_finite(rr)) {
      bad = 1;
    } else {
      const double rel = sqrt(rr / cur.bnorm2[c]);
      const double bta = rzn / cur.rz[c];  // computed alongside rel, kept only if not converged
      s->relres_inner[c] = rel;
      if (rel <= cur.inner_tol || !positive_finite(rzn)) {
        s->active[c] = 0;
        s->beta[c] = 0.0;
      } else {
        s->beta[c] = bta;
        s->rz[c] = rzn;
        act = 1;
      }
    }
  }
  const int nact = __popc(__ballot_sync(0xffffffffu, act));
  const int anybad = __any_sync(0xffffffffu, bad);
  int phase = kPhaseInner;
  if (c == 0) {
    const int it = cur.iter + 1, inner = cur.inner_iter + 1;
    s->iter = it;
    s->inner_iter = inner;
    if (anybad) {
      s->status = IG_ERR_NONFINITE;
      s->done = 1;
      phase = -1;
    } else if (nact == 0 || inner >= cur.inner_cap || it >= cur.max_iter) {
      s->phase = kPhaseApply;
      phase = kPhaseApply;
    }
  }
  return phase;
}

// ------------------------------------------------------------------------------- kernels
template <int K>
__global__ void __launch_bounds__(kBlock) init_mixed_kernel(const MeshDev* __restrict__ mds,
                                                            const int2* __restrict__ tiles, IoTable io, int rhs_mass,
                                                            LoopCtl* ctl, double tol, double inner_tol, int max_iter,
                                                            int max_refine, int cap) {
  __shared__ double sh[K * kBlock];
  const int2 tl = tiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const long nn = md.n;
  const long t0 = (long)tl.y * md.tile_rows32;
  const long t1 = t0 + md.tile_rows32 < nn ? t0 + md.tile_rows32 : nn;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->cnt = 0u;
    ctl->iter = 0;
    ctl->all_done = 0;
    ctl->any_apply = 0;
    ctl->ndone_start = 1 << 30;  // a whole solve stops only when every mesh is done
    ctl->cap = cap;
  }
  const double* __restrict__ src = io.in[tl.x];
  double acc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = 0.0;
  for (long base = t0; base < t1; base += kTileRows) {
#pragma unroll
    for (int rr = 0; rr < kRowsPerThread; ++rr) {
      const long row = base + rr * kBlock + threadIdx.x;
      if (row < t1) {
        const double mass = rhs_mass ? md.M[row] : 1.0;
#pragma unroll
        for (int c = 0; c < K; ++c) {
          const double b = rhs_mass ? mass * src[row * K + c] : src[row * K + c];
          md.rhs[c * nn + row] = b;
          md.r[c * nn + row] = b;
          md.x[c * nn + row] = 0.0;
          acc[c] = fma(b, b, acc[c]);
        }
      }
    }
  }
  if (reduce_tiles<K>(acc, md.part, tl.y, md.ntiles32, &md.s->cnt[2], sh) && threadIdx.x == 0)
    finish_init_mixed(md.s, K, acc, tol, inner_tol, max_iter, max_refine);
}

template <int K>
__global__ void __launch_bounds__(kBlock, 4) spmv_mixed_kernel(const MeshDev* __restrict__ mds, LoopCtl* ctl, ListRef L) {
  __shared__ TileCtx tc;
  tile_loop<K>(
      mds, L, 1, 0, tc, [](const ScalSnap& x) { return !x.done && x.phase == kPhaseInner; },
      [&](const MeshDev& md, int tile, double* red, double* out) {
        const long nn = md.n;
        const long t0 = (long)tile * md.tile_rows32;
        const long t1 = t0 + md.tile_rows32 < nn ? t0 + md.tile_rows32 : nn;
        const float* __restrict__ A = md.A32;
        const float* __restrict__ p = md.p32;
        float* __restrict__ q32 = md.q32;
        float pq[K];
#pragma unroll
        for (int c = 0; c < K; ++c) pq[c] = 0.f;
        // the SpMV's tiles have at most kTileRows rows: one pass
#pragma unroll
        for (int rr = 0; rr < kRowsPerThread; ++rr) {
          const long row = t0 + rr * kBlock + threadIdx.x;
          if (row < t1) {
            float q[K];
            row_product<K>(md, A, row, GatherP32<K>{p}, q);
            float pi[K];
            load_row32<K>(p, row, pi);
#pragma unroll
            for (int c = 0; c < K; ++c) {
              q32[c * nn + row] = q[c];
              pq[c] = fmaf(pi[c], q[c], pq[c]);
            }
          }
        }
        tile_reduce<K>(pq, red, out);
      },
      [](const MeshDev& md, const SolveScal& cur, const double* v) { finish_spmv(md.s, cur, K, v); });
}

// Apply phase: r64 = rhs - A64 x64 in FP64 and its squared norms (the refinement residual).
// Kept out of the FP32 SpMV kernel so that the hot FP32 kernel stays small; it walks the Apply
// list (the meshes in that phase), which the previous update launch built.
template <int K>
__global__ void __launch_bounds__(kBlock) resid_mixed_kernel(const MeshDev* __restrict__ mds, LoopCtl* ctl, ListRef L) {
  __shared__ TileCtx tc;
  if (!ctl->any_apply) return;  // no mesh of the group is in the Apply phase
  tile_loop<K>(
      mds, L, 1, 0, tc, [](const ScalSnap& x) { return !x.done && x.phase == kPhaseApply; },
      [&](const MeshDev& md, int tile, double* red, double* out) {
        const long nn = md.n;
        const long t0 = (long)tile * md.tile_rows32;
        const long t1 = t0 + md.tile_rows32 < nn ? t0 + md.tile_rows32 : nn;
        const double* __restrict__ x = md.x;
        const bool geom32 = md.geom32 != 0;  // the operator is the FP32 one: its values, exactly
        double acc[K];
#pragma unroll
        for (int c = 0; c < K; ++c) acc[c] = 0.0;
        // tiles of at most kTileRows rows: one pass
#pragma unroll
        for (int rr = 0; rr < kRowsPerThread; ++rr) {
          const long row = t0 + rr * kBlock + threadIdx.x;
          if (row < t1) {
            double ax[K];
            if (geom32) row_product<K>(md, md.A32, row, GatherSoA64<K>{x, nn}, ax);
            else row_product<K>(md, md.A, row, GatherSoA64<K>{x, nn}, ax);
#pragma unroll
            for (int c = 0; c < K; ++c) {
              const double res = md.rhs[c * nn + row] - ax[c];
              md.r[c * nn + row] = res;
              acc[c] = fma(res, res, acc[c]);
            }
          }
        }
        tile_reduce<K>(acc, red, out);
      },
      [](const MeshDev& md, const SolveScal& cur, const double* v) { finish_residual(md.s, cur, K, v); });
}

// Inner phase: x32 += alpha p32, r32 -= alpha q32 and the tile's sums r.z, r.r; all loads of a
// thread's rows are issued before its stores. Restart phase: r32 = r64 / ||r64||, x32 = 0.
template <int K>
__global__ void __launch_bounds__(kBlock, 4) update_mixed_kernel(const MeshDev* __restrict__ mds, LoopCtl* ctl, ListRef L,
    cudaGraphConditionalHandle handle, int use_graph) {
  __shared__ TileCtx tc;
  __shared__ int s_single, s_iter, s_cap, s_phase;
  if (threadIdx.x == 0) {
    s_single = (__ldcg(&ctl->nmesh) == 1);
    s_iter = __ldcg(&ctl->iter);
    s_cap = __ldcg(&ctl->cap);
    s_phase = kPhaseInner;
    tc.last = 0;
    // a group of one mesh that takes no part in this launch (done: its residual met the tolerance
    // in this iteration, or the loop stopped): no CTA completes it, so the loop is stopped here
    if (s_single && blockIdx.x == 0 && (__ldcg(&ctl->all_done) || __ldcg(&mds[0].s->done))) {
      ctl->all_done = 1;
      if (use_graph) cudaGraphSetConditional(handle, 0u);
    }
  }
  __syncthreads();
  tile_loop<2 * K>(
      mds, L, 2, 1, tc,
      [](const ScalSnap& x) { return !x.done && x.phase != kPhaseApply; },
      [&](const MeshDev& md, int tile, double* red, double* out) {
        const long nn = md.n;
        const long t0 = (long)tile * md.tile_rows32u;
        const long t1 = t0 + md.tile_rows32u < nn ? t0 + md.tile_rows32u : nn;
        PassSum<2 * K> sum;
        const float* __restrict__ D32 = md.Dinv32;
        float* __restrict__ x32 = md.x32;
        float* __restrict__ r32 = md.r32;
        if (tc.sn.phase == kPhaseInner) {
          const float* __restrict__ p32 = md.p32;
          const float* __restrict__ q32 = md.q32;
          const int n32 = md.n;
          float alpha[K];
#pragma unroll
          for (int c = 0; c < K; ++c) alpha[c] = (float)tc.sn.alpha[c];
          constexpr int RB = 2;
          for (long base = t0; base < t1; base += kTileRows) {
            float acc[2 * K];
#pragma unroll
            for (int i = 0; i < 2 * K; ++i) acc[i] = 0.f;
#pragma unroll
            for (int r0 = 0; r0 < kRowsPerThread; r0 += RB) {
              float d[RB], pi[RB][K], xs[RB][K], qs[RB][K], rs[RB][K];
#pragma unroll
              for (int u = 0; u < RB; ++u) {
                const int row = (int)base + (r0 + u) * kBlock + threadIdx.x;
                if (row < (int)t1) {
                  d[u] = D32[row];
                  load_row32<K>(p32, row, pi[u]);
#pragma unroll
                  for (int c = 0; c < K; ++c) {
                    xs[u][c] = x32[(long)c * n32 + row];
                    qs[u][c] = q32[(long)c * n32 + row];
                    rs[u][c] = r32[(long)c * n32 + row];
                  }
                }
              }
#pragma unroll
              for (int u = 0; u < RB; ++u) {
                const int row = (int)base + (r0 + u) * kBlock + threadIdx.x;
                if (row < (int)t1) {
#pragma unroll
                  for (int c = 0; c < K; ++c) {
                    const float rv = fmaf(-alpha[c], qs[u][c], rs[u][c]);
                    x32[(long)c * n32 + row] = fmaf(alpha[c], pi[u][c], xs[u][c]);
                    r32[(long)c * n32 + row] = rv;
                    acc[c] = fmaf(rv, d[u] * rv, acc[c]);
                    acc[K + c] = fmaf(rv, rv, acc[K + c]);
                  }
                }
              }
            }
            sum.add(acc);
          }
        } else {
          // Restart: r32 = r64 / ||r64|| for columns still above tol, d = 0
          double inv[K];
          int act[K];
#pragma unroll
          for (int c = 0; c < K; ++c) {
            act[c] = tc.sn.act64[c];
            inv[c] = 1.0 / tc.sn.scale[c];
          }
          const double* __restrict__ r64 = md.r;
          for (long base = t0; base < t1; base += kTileRows) {
            float acc[2 * K];
#pragma unroll
            for (int i = 0; i < 2 * K; ++i) acc[i] = 0.f;
#pragma unroll
            for (int rr = 0; rr < kRowsPerThread; ++rr) {
              const long row = base + rr * kBlock + threadIdx.x;
              if (row < t1) {
                const float dinv = D32[row];
#pragma unroll
                for (int c = 0; c < K; ++c) {
                  const float rv = act[c] ? (float)(r64[c * nn + row] * inv[c]) : 0.f;
                  r32[c * nn + row] = rv;
                  x32[c * nn + row] = 0.f;
                  acc[c] = fmaf(rv, dinv * rv, acc[c]);
                  acc[K + c] = fmaf(rv, rv, acc[K + c]);
                }
              }
            }
            sum.add(acc);
          }
        }
        tile_reduce<2 * K>(sum.s, red, out);
      },
      [&](const MeshDev& md, const SolveScal& cur, const double* v) {
        const int phase = cur.phase == kPhaseInner ? finish_update_mixed(md.s, cur, K, v)
                                                   : finish_restart(md.s, cur, K, v);
        if (threadIdx.x == 0) s_phase = phase;
      });
  if (!s_single) {
    loop_control(mds, ctl, handle, use_graph);
  } else if (tc.last) {
    // the CTA that completed the mesh (flush_tiles ended in a barrier, so s_phase is visible): the
    // next iteration recomputes the FP64 residual when the inner solve just ended; the Apply list
    // is rebuilt by the whole CTA
    const int apply = s_phase == kPhaseApply;
    if (apply && ctl->app_mesh) rebuild_apply(mds, ctl);
    if (threadIdx.x == 0) {
      ctl->any_apply = apply;
      single_loop_control(s_phase < 0, s_iter, s_cap, ctl, handle, use_graph);
    }
  }
}

// Inner phase: p32 = D^-1 r32 + beta p32 (loads of a thread's rows before its stores). Apply
// phase: x64 += ||r64|| x32.
template <int K>
// In the graph loop of a single mesh (use_graph), CTA 0 also sets the condition of the IF node that
// holds the next iteration's residual kernel: whether the mesh recomputes its FP64 residual then
// (any_apply, as the update launch before this one left it). Iterations without a refinement so
// skip that launch.
__global__ void __launch_bounds__(kBlock, 4) pupdate_mixed_kernel(const MeshDev* __restrict__ mds, LoopCtl* ctl, ListRef L,
                                                                  cudaGraphConditionalHandle apply_handle,
                                                                  int use_graph) {
  __shared__ TileCtx tc;
  if (use_graph && blockIdx.x == 0 && threadIdx.x == 0)
    cudaGraphSetConditional(apply_handle, __ldcg(&ctl->any_apply) ? 1u : 0u);
  tile_loop_plain(mds, L, 1, tc,
                  [](const ScalSnap& x) { return !x.done && (x.phase == kPhaseInner || x.phase == kPhaseApply); },
                  [&](const MeshDev& md, int tile) {
                    const long nn = md.n;
                    const long t0 = (long)tile * md.tile_rows32;
                    const long t1 = t0 + md.tile_rows32 < nn ? t0 + md.tile_rows32 : nn;
                    if (tc.sn.phase == kPhaseInner) {
                      float beta[K];
#pragma unroll
                      for (int c = 0; c < K; ++c) beta[c] = (float)tc.sn.beta[c];
                      const float* __restrict__ D32 = md.Dinv32;
                      const float* __restrict__ r32 = md.r32;
                      float* __restrict__ p32 = md.p32;
                      constexpr int R = kRowsPerThread;  // one pass: tiles of at most kTileRows rows
                      float d[R], pi[R][K], rs[R][K];
#pragma unroll
                      for (int u = 0; u < R; ++u) {
                        const long row = t0 + u * kBlock + threadIdx.x;
                        if (row < t1) {
                          d[u] = D32[row];
                          load_row32<K>(p32, row, pi[u]);
#pragma unroll
                          for (int c = 0; c < K; ++c) rs[u][c] = r32[c * nn + row];
                        }
                      }
#pragma unroll
                      for (int u = 0; u < R; ++u) {
                        const long row = t0 + u * kBlock + threadIdx.x;
                        if (row < t1) {
#pragma unroll
                          for (int c = 0; c < K; ++c)
                            p32[row * KPm<K>::v + c] = fmaf(beta[c], pi[u][c], d[u] * rs[u][c]);
                        }
                      }
                    } else {
                      double sc[K];
#pragma unroll
                      for (int c = 0; c < K; ++c) sc[c] = tc.sn.scale[c];
                      const float* __restrict__ x32 = md.x32;
                      double* __restrict__ x = md.x;
#pragma unroll
                      for (int rr = 0; rr < kRowsPerThread; ++rr) {
                        const long row = t0 + rr * kBlock + threadIdx.x;
                        if (row < t1) {
#pragma unroll
                          for (int c = 0; c < K; ++c)
                            x[c * nn + row] = fma(sc[c], (double)x32[c * nn + row], x[c * nn + row]);
                        }
                      }
                    }
                  });
}

template <int K>
cudaError_t build_plan_mixed(Group& g, SolvePlan& pl) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle handle;
  e = cudaGraphConditionalHandleCreate(&handle, graph, 1u, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) { cudaGraphDestroy(graph); return e; }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  if (e != cudaSuccess) { cudaGraphDestroy(graph); return e; }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t cs = g.capture_stream;
  // A group of one mesh: the body is an IF node holding the residual kernel (its condition set by
  // the p-update of the iteration before; the value it starts a solve with is irrelevant, since no
  // mesh recomputes its residual in a solve's first iteration and the kernel itself returns when
  // none does), then the SpMV, the update and the p-update. A group of many meshes has some mesh
  // refining in most iterations, where the IF node costs more than it saves: its body launches the
  // residual kernel every iteration.
  const bool use_if = g.nmesh == 1;
  cudaGraphConditionalHandle apply_handle{};
  cudaGraphNode_t if_node = nullptr;
  cudaGraph_t captured = nullptr;
  cudaError_t le = cudaSuccess;
  if (use_if) {
    e = cudaGraphConditionalHandleCreate(&apply_handle, body, 1u, 0u);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return e; }
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = apply_handle;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    e = cudaGraphAddNode(&if_node, body, nullptr, nullptr, 0, &ip);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return e; }
    cudaGraph_t resid_body = ip.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cs, resid_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return e; }
    resid_mixed_kernel<K><<<g.grid32, kBlock, 0, cs>>>(g.mds, g.ctl, g.listapp);
    le = cudaGetLastError();
    e = cudaStreamEndCapture(cs, &captured);
    if (le != cudaSuccess) e = le;
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return e; }
    e = cudaStreamBeginCaptureToGraph(cs, body, &if_node, nullptr, 1, cudaStreamCaptureModeThreadLocal);
  } else {
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  }
  if (e != cudaSuccess) { cudaGraphDestroy(graph); return e; }
  if (!use_if) resid_mixed_kernel<K><<<g.grid32, kBlock, 0, cs>>>(g.mds, g.ctl, g.listapp);
  spmv_mixed_kernel<K><<<g.grid32, kBlock, 0, cs>>>(g.mds, g.ctl, g.list32);
  update_mixed_kernel<K><<<g.grid32, kBlock, 0, cs>>>(g.mds, g.ctl, g.list32, handle, 1);
  pupdate_mixed_kernel<K><<<g.grid32, kBlock, 0, cs>>>(g.mds, g.ctl, g.list32, apply_handle, use_if ? 1 : 0);
  le = cudaGetLastError();
  e = cudaStreamEndCapture(cs, &captured);
  if (le != cudaSuccess) e = le;
  if (e != cudaSuccess) { cudaGraphDestroy(graph); return e; }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) { cudaGraphDestroy(graph); return e; }
  pl.k = K;
  pl.mixed = 1;
  pl.graph = graph;
  pl.exec = exec;
  return cudaSuccess;
}

template <int K>
cudaError_t begin_mixed_k(Group& g, const IoTable& io, int rhs_mass, const ig_solve_opts& o, cudaStream_t st) {
  const int cap = o.max_iter + 3 * o.max_refine + 4;
  IG_PROF("pcg_init", st);
  init_mixed_kernel<K><<<g.ntiles32, kBlock, 0, st>>>(g.mds, g.tiles32, io, rhs_mass, g.ctl, o.rel_tol, o.inner_tol,
                                                      o.max_iter, o.max_refine, cap);
  list_kernel<<<1, kBlock, 0, st>>>(g.mds, g.ctl);
  return cudaGetLastError();
}

template <int K>
cudaError_t host_loop_mixed_k(Group& g, int max_it, int poll, cudaStream_t st) {
  cudaError_t e;
  for (int it = 0; it < max_it; ++it) {
    {
      IG_PROF("pcg32_resid64", st);
      resid_mixed_kernel<K><<<g.grid32, kBlock, 0, st>>>(g.mds, g.ctl, g.listapp);
    }
    {
      IG_PROF("pcg32_spmv", st);
      spmv_mixed_kernel<K><<<g.grid32, kBlock, 0, st>>>(g.mds, g.ctl, g.list32);
    }
    {
      IG_PROF("pcg32_update", st);
      update_mixed_kernel<K><<<g.grid32, kBlock, 0, st>>>(g.mds, g.ctl, g.list32, cudaGraphConditionalHandle{}, 0);
    }
    {
      IG_PROF("pcg32_pupdate", st);
      pupdate_mixed_kernel<K><<<g.grid32, kBlock, 0, st>>>(g.mds, g.ctl, g.list32, cudaGraphConditionalHandle{}, 0);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (prof_on() || (it % poll) == poll - 1 || it == max_it - 1) {
      e = cudaMemcpyAsync(g.done_host, &g.ctl->all_done, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return e;
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return e;
      if (*g.done_host) break;
    }
  }
  return cudaSuccess;
}

template <int K>
cudaError_t solve_mixed_k(Group& g, const IoTable& io, int rhs_mass, const ig_solve_opts& o, cudaStream_t st) {
  cudaError_t e = begin_mixed_k<K>(g, io, rhs_mass, o, st);
  if (e != cudaSuccess) return e;
  if (o.launch == IG_LAUNCH_GRAPH && !prof_on()) {
    SolvePlan& pl = g.plans[1][K];
    if (!pl.exec) {
      e = build_plan_mixed<K>(g, pl);
      if (e != cudaSuccess) return e;
    }
    e = cudaGraphLaunch(pl.exec, st);
  } else {
    e = host_loop_mixed_k<K>(g, o.max_iter + 3 * o.max_refine + 4, 16, st);
  }
  if (e != cudaSuccess) return e;
  IG_PROF("pcg_finalize", st);
  finalize_kernel<K><<<g.ntiles, kBlock, 0, st>>>(g.mds, g.tiles, io);
  return cudaGetLastError();
}

}  // namespace

int solver_blocks_per_sm_mixed() {
  int a = 0, b = 0, c = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, spmv_mixed_kernel<3>, kBlock, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, update_mixed_kernel<3>, kBlock, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, pupdate_mixed_kernel<3>, kBlock, 0);
  int m = a < b ? a : b;
  m = m < c ? m : c;
  return m > 0 ? m : 1;
}

cudaError_t group_begin_mixed(Group& g, int k, const IoTable& io, int rhs_mass, const ig_solve_opts& o,
                              cudaStream_t st) {
  switch (k) {
    case 1: return begin_mixed_k<1>(g, io, rhs_mass, o, st);
    case 2: return begin_mixed_k<2>(g, io, rhs_mass, o, st);
    case 3: return begin_mixed_k<3>(g, io, rhs_mass, o, st);
    case 4: return begin_mixed_k<4>(g, io, rhs_mass, o, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t group_host_loop_mixed(Group& g, int k, int budget, cudaStream_t st) {
  switch (k) {
    case 1: return host_loop_mixed_k<1>(g, budget, 8, st);
    case 2: return host_loop_mixed_k<2>(g, budget, 8, st);
    case 3: return host_loop_mixed_k<3>(g, budget, 8, st);
    case 4: return host_loop_mixed_k<4>(g, budget, 8, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t group_solve_mixed(Group& g, int k, const IoTable& io, int rhs_mass, const ig_solve_opts& o,
                              cudaStream_t st) {
  switch (k) {
    case 1: return solve_mixed_k<1>(g, io, rhs_mass, o, st);
    case 2: return solve_mixed_k<2>(g, io, rhs_mass, o, st);
    case 3: return solve_mixed_k<3>(g, io, rhs_mass, o, st);
    case 4: return solve_mixed_k<4>(g, io, rhs_mass, o, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ig
