// ig_pcg.cu -- Jacobi-preconditioned conjugate gradients for A X = RHS with k <= 4 columns
// solved together (the matrix is read once per iteration for all columns), on a group of one or
// more meshes (the forward solve of §7.1 and the adjoint solve of §5.2 use the same operator).
//
// One iteration is two kernels over tiles of up to kTileRows64 rows (a tile belongs to one mesh):
//   spmv   : p = z + beta p, q = A p = A z + beta q (the product carried by its recurrence, so
//            that the direction update needs no pass of its own), partial p.q
//            -> last tile of the mesh: alpha = rz / pq
//   update : x += alpha p, r -= alpha q, z = D^-1 r, partial r.z and r.r
//            -> last tile of the mesh: convergence test, beta = rz_new / rz
//            -> last CTA of the launch: loop control (all meshes done or the cap reached)
// Reductions are deterministic: every CTA writes its partial sums, the last CTA of a mesh (found
// with a counter) adds the partials in tile order. No atomics touch floating-point data, so a mesh
// gives the same bits alone and inside a batch.
//
// The loop runs on the device: a CUDA graph holds a WHILE node whose body is one iteration; the
// update kernel's last CTA clears the condition when the group is done, so the host neither
// polls nor synchronises per iteration. Every loop is bounded by a hard cap.
//
// FP64 instructions are the scarce resource of this GPU (2 FP64 FMA per clock per SM). Each thread
// handles several rows of a tile so the block reductions, which cost FP64 adds, are amortised.
#include <cstring>
#include <mutex>

#include "ig_device.cuh"

namespace ig {

namespace {

// ------------------------------------------------------------------------------- last-CTA steps
// The per-mesh scalar updates run on one thread of the last CTA of a reduction. They are kept
// out of line (and count active columns explicitly) so that this bookkeeping is compiled on its
// own, apart from the unrolled arithmetic of the kernels.
__device__ __noinline__ void finish_init(SolveScal* s, int k, const double* acc, double tol, int max_iter) {
  int nact = 0, bad = 0;
  for (int c = 0; c < kMaxK; ++c) {
    const double rz = c < k ? acc[c] : 0.0;
    const double bb = c < k ? acc[k + c] : 0.0;
    if (c < k && (!is_finite(bb) || !is_finite(rz))) bad = 1;
    const int act = (c < k && positive_finite(bb)) ? 1 : 0;
    s->rz[c] = rz;
    s->bnorm2[c] = bb;
    s->rhs2[c] = bb;
    s->active[c] = act;
    s->relres[c] = act ? 1.0 : 0.0;
    s->alpha[c] = 0.0;
    s->beta[c] = 0.0;
    s->scale[c] = 1.0;
    s->trueres[c] = -1.0;
    nact += act;
  }
  s->k = k;
  s->cnt[0] = 0u;
  s->cnt[1] = 0u;
  s->iter = 0;
  s->refine = 0;
  s->phase = 0;
  s->tol = tol;
  s->max_iter = max_iter;
  s->status = bad ? IG_ERR_NONFINITE : IG_OK;
  s->done = (bad != 0 || nact == 0) ? 1 : 0;
}

// Convergence test per column (recursive residual), beta_c = rz_new / rz, iteration count. Runs on
// warp 0 of the CTA that completes the mesh: lane c takes column c, lane 0 the mesh's fields.
// Returns (on lane 0) whether the mesh is now done.
__device__ __noinline__ int finish_update(SolveScal* s, const SolveScal& cur, int k, const double* acc) {
  const int c = threadIdx.x & 31;
  int act = 0, bad = 0;
  if (c < k && cur.active[c] != 0) {
    const double rzn = acc[c], rr = acc[k + c];
    if (!is_finite(rzn) || !is_finite(rr)) {
      bad = 1;
    } else {
      const double rel = sqrt(rr / cur.bnorm2[c]);
      const double bta = rzn / cur.rz[c];  // computed alongside rel, kept only if not converged
      s->relres[c] = rel;
      if (rel <= cur.tol) {
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
  int done = 0;
  if (c == 0) {
    const int it = cur.iter + 1;
    s->iter = it;
    if (anybad) {
      s->status = IG_ERR_NONFINITE;
      done = 1;
    } else if (nact == 0) {
      done = 1;
    } else if (it >= cur.max_iter) {
      s->status = IG_ERR_NOT_CONVERGED;
      done = 1;
    }
    if (done) s->done = 1;
  }
  return done;
}

// ------------------------------------------------------------------------------- init
// rhs = M * in (rhs_mass) or in; x = 0; r = rhs; z = D^-1 r; p = q = 0; per mesh: rz, ||rhs||^2.
template <int K>
__global__ void __launch_bounds__(kBlock) init_kernel(const MeshDev* __restrict__ mds, const int2* __restrict__ tiles,
                                                      IoTable io, int rhs_mass, LoopCtl* ctl, double tol,
                                                      int max_iter, int cap) {
  __shared__ double sh[2 * K * kBlock];
  const int2 tl = tiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const long nn = md.n;
  const long t0 = (long)tl.y * md.tile_rows;
  const long t1 = t0 + md.tile_rows < nn ? t0 + md.tile_rows : nn;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->cnt = 0u;
    ctl->iter = 0;
    ctl->all_done = 0;
    ctl->any_apply = 0;
    ctl->ndone_start = 1 << 30;  // a whole solve stops only when every mesh is done
    ctl->cap = cap;
  }
  const double* __restrict__ src = io.in[tl.x];
  double acc[2 * K];
#pragma unroll
  for (int i = 0; i < 2 * K; ++i) acc[i] = 0.0;
  for (long row = t0 + threadIdx.x; row < t1; row += kBlock) {
    const double dinv = md.Dinv[row];
    const double mass = rhs_mass ? md.M[row] : 1.0;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const double b = rhs_mass ? mass * src[row * K + c] : src[row * K + c];
      const double z = dinv * b;
      md.x[c * nn + row] = 0.0;
      md.r[c * nn + row] = b;
      md.z[row * KP<K>::v + c] = z;
      md.p[row * KP<K>::v + c] = 0.0;  // with beta = 0 the first SpMV sets p = z, q = A z
      md.q[c * nn + row] = 0.0;
      acc[c] = fma(b, z, acc[c]);
      acc[K + c] = fma(b, b, acc[K + c]);
    }
  }
  if (reduce_tiles<2 * K>(acc, md.part, tl.y, md.ntiles, &md.s->cnt[2], sh) && threadIdx.x == 0)
    finish_init(md.s, K, acc, tol, max_iter);
}

// ------------------------------------------------------------------------------- spmv
// The search direction and its product with A in one pass, for the rows of one tile (t0..t1):
// p = z + beta p and q = A p = A z + beta q (z = D^-1 r from the update kernel; A z gathers z),
// and the tile's sums p.q. Carrying q = A p by this recurrence removes the separate p-update
// pass of the textbook iteration (its p = z + beta p happens here), so an iteration is two
// kernels. beta = 0 at the start of a solve (p = q = 0 there), so the first pass is q = A z.
template <int K>
__device__ __forceinline__ void spmv_tile(const MeshDev& md, int tile, const ScalSnap& sn, double* red,
                                          double* out) {
  const long nn = md.n;
  const long t0 = (long)tile * md.tile_rows;
  const long t1 = t0 + md.tile_rows < nn ? t0 + md.tile_rows : nn;
  const double* __restrict__ A = md.A;
  const double* __restrict__ z = md.z;
  double* __restrict__ p = md.p;
  double* __restrict__ q = md.q;
  double pq[K];
#pragma unroll
  for (int c = 0; c < K; ++c) pq[c] = 0.0;
  for (long row = t0 + threadIdx.x; row < t1; row += kBlock) {
    double w[K];
    row_product<K>(md, A, row, GatherP64<K>{z}, w);
    double zi[K], pi[K], qi[K];
    load_row<K>(z, row, zi);
    load_row<K>(p, row, pi);
#pragma unroll
    for (int c = 0; c < K; ++c) qi[c] = q[c * nn + row];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const double b = sn.beta[c];
      const double pn = fma(b, pi[c], zi[c]);
      const double qn = fma(b, qi[c], w[c]);
      p[row * KP<K>::v + c] = pn;
      q[c * nn + row] = qn;
      pq[c] = fma(pn, qn, pq[c]);
    }
  }
  tile_reduce<K>(pq, red, out);
}

template <int K>
__global__ void __launch_bounds__(kBlock, 4) spmv_kernel(const MeshDev* __restrict__ mds, LoopCtl* ctl, ListRef L) {
  __shared__ TileCtx tc;
  __shared__ int s_stop;  // the loop has stopped: a launch after that (second half of a graph pass) does nothing
  if (threadIdx.x == 0) s_stop = __ldcg(&ctl->all_done);
  tile_loop<K>(
      mds, L, 0, 0, tc, [&](const ScalSnap& x) { return !x.done && !s_stop; },
      [&](const MeshDev& md, int tile, double* red, double* out) { spmv_tile<K>(md, tile, tc.sn, red, out); },
      [](const MeshDev& md, const SolveScal& cur, const double* v) { finish_spmv(md.s, cur, K, v); });
}

// ------------------------------------------------------------------------------- update
// x += alpha p, r -= alpha q, z = D^-1 r (rows padded like p, for the next SpMV's gathers) and the
// tile's sums r.z, r.r; a row's loads are issued before its stores. Rows are taken one at a time:
// FP64 arithmetic bounds this kernel, and unrolling the row loop only spills at 64 registers.
template <int K>
__device__ __forceinline__ void update_tile(const MeshDev& md, int tile, const ScalSnap& sn, double* red,
                                            double* out) {
  const int nn = md.n;
  const int t0 = tile * md.tile_rows;
  const int t1 = t0 + md.tile_rows < nn ? t0 + md.tile_rows : nn;
  double acc[2 * K];
#pragma unroll
  for (int i = 0; i < 2 * K; ++i) acc[i] = 0.0;
  const double* __restrict__ Dinv = md.Dinv;
  const double* __restrict__ p = md.p;
  const double* __restrict__ q = md.q;
  double* __restrict__ zv = md.z;
  double* __restrict__ x = md.x;
  double* __restrict__ r = md.r;
#pragma unroll 1
  for (int row = t0 + threadIdx.x; row < t1; row += kBlock) {
    double pi[K], xs[K], qs[K], rs[K];
    const double d = Dinv[row];
    load_row<K>(p, row, pi);
#pragma unroll
    for (int c = 0; c < K; ++c) {
      xs[c] = x[(long)c * nn + row];
      qs[c] = q[(long)c * nn + row];
      rs[c] = r[(long)c * nn + row];
    }
    double zo[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const double a = sn.alpha[c];
      const double rn = fma(-a, qs[c], rs[c]);
      zo[c] = d * rn;
      x[(long)c * nn + row] = fma(a, pi[c], xs[c]);
      r[(long)c * nn + row] = rn;
      acc[c] = fma(rn, zo[c], acc[c]);
      acc[K + c] = fma(rn, rn, acc[K + c]);
    }
    store_row<K>(zv, row, zo);
  }
  tile_reduce<2 * K>(acc, red, out);
}

template <int K>
__global__ void __launch_bounds__(kBlock, 4) update_kernel(const MeshDev* __restrict__ mds, LoopCtl* ctl, ListRef L,
    cudaGraphConditionalHandle handle, int use_graph) {
  __shared__ TileCtx tc;
  __shared__ int s_single, s_stop, s_iter, s_cap, s_done;
  if (threadIdx.x == 0) {
    s_single = (__ldcg(&ctl->nmesh) == 1);
    s_stop = __ldcg(&ctl->all_done);
    s_iter = __ldcg(&ctl->iter);
    s_cap = __ldcg(&ctl->cap);
    s_done = 0;
    // a group of one mesh whose mesh takes no part in this launch (done, or the loop stopped):
    // no CTA completes it, so the loop is stopped here
    if (s_single && blockIdx.x == 0 && (s_stop || __ldcg(&mds[0].s->done))) {
      ctl->all_done = 1;
      if (use_graph) cudaGraphSetConditional(handle, 0u);
    }
  }
  if (threadIdx.x == 0) tc.last = 0;
  __syncthreads();
  tile_loop<2 * K>(
      mds, L, 0, 1, tc, [&](const ScalSnap& x) { return !x.done && !s_stop; },
      [&](const MeshDev& md, int tile, double* red, double* out) { update_tile<K>(md, tile, tc.sn, red, out); },
      [&](const MeshDev& md, const SolveScal& cur, const double* v) {
        const int done = finish_update(md.s, cur, K, v);
        if (threadIdx.x == 0) s_done = done;
      });
  if (!s_single) {
    loop_control(mds, ctl, handle, use_graph);
  } else if (tc.last && threadIdx.x == 0) {
    // the CTA that completed the mesh (its finish step is done: flush_tiles ends in a barrier)
    single_loop_control(s_done, s_iter, s_cap, ctl, handle, use_graph);
  }
}

// ------------------------------------------------------------------------------- small meshes
// The whole iteration loop of a small single mesh (at most kSmallTiles FP64 tiles) in one
// thread-block cluster with one CTA per tile. A CTA runs its tile through the tile bodies of the
// multi-CTA kernels and publishes the tile's partial sums; after a cluster barrier every CTA adds
// all the partials in tile order and runs the finish step on its own shared-memory copy of the
// solve state (the same inputs and arithmetic in every CTA, so the copies stay equal), and goes
// on. Two cluster barriers per iteration replace the kernel boundaries, the last-CTA hand-offs
// and the graph loop's node transitions, which make up most of an iteration of a mesh of a few
// tiles. The arithmetic and its order are those of the multi-CTA path: the same bits. The SpMV's
// and the update's partials live in separate halves of the partial buffer, so a CTA that runs
// ahead never overwrites partials that another CTA is still adding.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int NV, typename Finish>
__device__ __forceinline__ void finish_cluster(TileCtx& tc, SolveScal& st, const double* part, int nt,
                                               const Finish& finish) {
  double v[NV];
  gather_partials<NV>(part, nt, v);
  if (threadIdx.x < (int)(sizeof(SolveScal) / 4))
    reinterpret_cast<unsigned*>(&tc.cur)[threadIdx.x] = reinterpret_cast<const unsigned*>(&st)[threadIdx.x];
  tile_reduce<NV>(v, tc.red[0], tc.tot);
  __syncthreads();
  if (threadIdx.x < 32) finish(&st, tc.cur, tc.tot);
  __syncthreads();
}

template <int K>
__global__ void __launch_bounds__(kBlock) solve_cluster_kernel(const MeshDev* __restrict__ mds, LoopCtl* ctl) {
  __shared__ TileCtx tc;
  __shared__ SolveScal st;
  load_mesh(mds, 0, tc);
  const int nt = tc.md.ntiles, tile = blockIdx.x;
  static_assert(sizeof(SolveScal) % 4 == 0 && sizeof(SolveScal) / 4 <= kBlock, "SolveScal copy");
  if (threadIdx.x < (int)(sizeof(SolveScal) / 4))
    reinterpret_cast<unsigned*>(&st)[threadIdx.x] = __ldcg(reinterpret_cast<const unsigned*>(tc.md.s) + threadIdx.x);
  __syncthreads();
  double* part_spmv = tc.md.part;
  double* part_upd = tc.md.part + (long)nt * kPartStride;
  const int cap = __ldcg(&ctl->cap);
  int it = 0;
  for (; it < cap && !st.done; ++it) {
    if (threadIdx.x < kMaxK) tc.sn.beta[threadIdx.x] = st.beta[threadIdx.x];
    __syncthreads();
    spmv_tile<K>(tc.md, tile, tc.sn, tc.red[1], part_spmv + (long)tile * kPartStride);
    cluster_sync_all();
    finish_cluster<K>(tc, st, part_spmv, nt,
                      [](SolveScal* s, const SolveScal& cur, const double* v) { finish_spmv(s, cur, K, v); });
    if (threadIdx.x < kMaxK) tc.sn.alpha[threadIdx.x] = st.alpha[threadIdx.x];
    __syncthreads();
    update_tile<K>(tc.md, tile, tc.sn, tc.red[1], part_upd + (long)tile * kPartStride);
    cluster_sync_all();
    finish_cluster<2 * K>(tc, st, part_upd, nt,
                          [](SolveScal* s, const SolveScal& cur, const double* v) { finish_update(s, cur, K, v); });
  }
  if (blockIdx.x == 0) {
    if (threadIdx.x < (int)(sizeof(SolveScal) / 4))
      reinterpret_cast<unsigned*>(tc.md.s)[threadIdx.x] = reinterpret_cast<const unsigned*>(&st)[threadIdx.x];
    if (threadIdx.x == 0) {
      ctl->iter = it;
      ctl->all_done = 1;
    }
  }
}

// Launch of the cluster loop: one cluster of ntiles CTAs (non-portable sizes above 8 allowed).
// Returns false, with nothing launched, when the device refuses that cluster.
template <int K>
bool launch_cluster_loop(Group& g, cudaStream_t st) {
  const int nt = g.host_mds[0].ntiles;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(solve_cluster_kernel<K>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
        cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nt, 1, 1);
  cfg.blockDim = dim3(kBlock, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nt;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, solve_cluster_kernel<K>, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return false;
  }
  if (cudaLaunchKernelEx(&cfg, solve_cluster_kernel<K>, (const MeshDev*)g.mds, g.ctl) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// ------------------------------------------------------------------------------- true residual
// trueres = ||rhs - A x|| / ||rhs|| per column with x = io.out (the written solution).
template <int K>
__global__ void __launch_bounds__(kBlock) residual_kernel(const MeshDev* __restrict__ mds,
                                                          const int2* __restrict__ tiles, IoTable io, int rhs_mass) {
  __shared__ double sh[K * kBlock];
  const int2 tl = tiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const long nn = md.n;
  const long t0 = (long)tl.y * md.tile_rows;
  const long t1 = t0 + md.tile_rows < nn ? t0 + md.tile_rows : nn;
  const double* __restrict__ src = io.in[tl.x];
  const double* __restrict__ xs = io.out[tl.x];
  double acc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = 0.0;
  for (long row = t0 + threadIdx.x; row < t1; row += kBlock) {
    double ax[K];
    if (md.geom32) row_product<K>(md, md.A32, row, GatherAoS64<K>{xs}, ax);  // the FP32 operator, exactly
    else row_product<K>(md, md.A, row, GatherAoS64<K>{xs}, ax);
    const double mass = rhs_mass ? md.M[row] : 1.0;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const double b = rhs_mass ? mass * src[row * K + c] : src[row * K + c];
      const double res = b - ax[c];
      acc[c] = fma(res, res, acc[c]);
    }
  }
  if (reduce_tiles<K>(acc, md.part, tl.y, md.ntiles, &md.s->cnt[2], sh) && threadIdx.x == 0) {
    for (int c = 0; c < K; ++c) {
      const double r2 = md.s->rhs2[c];
      md.s->trueres[c] = r2 > 0.0 ? sqrt(acc[c] / r2) : sqrt(acc[c]);
    }
  }
}

template <int K>
cudaError_t build_plan(Group& g, SolvePlan& pl) {
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
  e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaGraphDestroy(graph); return e; }
  // Two iterations per pass of the WHILE body: its re-evaluation costs more than a kernel
  // boundary. When the first iteration ends the loop, the second pair of launches finds every
  // mesh done and returns at once.
  for (int u = 0; u < 2; ++u) {
    spmv_kernel<K><<<g.grid64, kBlock, 0, cs>>>(g.mds, g.ctl, g.list64);
    update_kernel<K><<<g.grid64, kBlock, 0, cs>>>(g.mds, g.ctl, g.list64, handle, 1);
  }
  cudaError_t le = cudaGetLastError();
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(cs, &captured);
  if (le != cudaSuccess) e = le;
  if (e != cudaSuccess) { cudaGraphDestroy(graph); return e; }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) { cudaGraphDestroy(graph); return e; }
  pl.k = K;
  pl.mixed = 0;
  pl.graph = graph;
  pl.exec = exec;
  return cudaSuccess;
}

template <int K>
cudaError_t begin_k(Group& g, const IoTable& io, int rhs_mass, const ig_solve_opts& o, cudaStream_t st) {
  const int cap = o.max_iter + 2;
  IG_PROF("pcg_init", st);
  init_kernel<K><<<g.ntiles, kBlock, 0, st>>>(g.mds, g.tiles, io, rhs_mass, g.ctl, o.rel_tol, o.max_iter, cap);
  list_kernel<<<1, kBlock, 0, st>>>(g.mds, g.ctl);
  return cudaGetLastError();
}

// Host-driven loop: up to max_it iterations, polling the device's stop word every `poll`.
template <int K>
cudaError_t host_loop_k(Group& g, int max_it, int poll, cudaStream_t st) {
  cudaError_t e;
  for (int it = 0; it < max_it; ++it) {
    {
      IG_PROF("pcg_spmv", st);
      spmv_kernel<K><<<g.grid64, kBlock, 0, st>>>(g.mds, g.ctl, g.list64);
    }
    {
      IG_PROF("pcg_update", st);
      update_kernel<K><<<g.grid64, kBlock, 0, st>>>(g.mds, g.ctl, g.list64, cudaGraphConditionalHandle{}, 0);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // poll every `poll` iterations (every iteration while kernels are being timed, so that no
    // launch after convergence is timed)
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
cudaError_t loop_k(Group& g, const ig_solve_opts& o, cudaStream_t st) {
  if (o.launch == IG_LAUNCH_GRAPH && !prof_on() && g.nmesh == 1 && g.host_mds[0].ntiles <= kSmallTiles &&
      launch_cluster_loop<K>(g, st))
    return cudaSuccess;
  if (o.launch == IG_LAUNCH_GRAPH && !prof_on()) {
    SolvePlan& pl = g.plans[0][K];
    if (!pl.exec) {
      cudaError_t e = build_plan<K>(g, pl);
      if (e != cudaSuccess) return e;
    }
    return cudaGraphLaunch(pl.exec, st);
  }
  return host_loop_k<K>(g, o.max_iter + 2, 16, st);
}

template <int K>
cudaError_t end_k(Group& g, const IoTable& io, cudaStream_t st) {
  IG_PROF("pcg_finalize", st);
  finalize_kernel<K><<<g.ntiles, kBlock, 0, st>>>(g.mds, g.tiles, io);
  return cudaGetLastError();
}

template <int K>
cudaError_t solve_k(Group& g, const IoTable& io, int rhs_mass, const ig_solve_opts& o, cudaStream_t st) {
  cudaError_t e = begin_k<K>(g, io, rhs_mass, o, st);
  if (e == cudaSuccess) e = loop_k<K>(g, o, st);
  if (e == cudaSuccess) e = end_k<K>(g, io, st);
  return e;
}

// Serving: restart the loop counters of a group whose members may be mid-solve. The loop stops
// after `budget` iterations, or as soon as a member that was running has finished.
__global__ void __launch_bounds__(kBlock) loop_reset_kernel(const MeshDev* __restrict__ mds, LoopCtl* ctl,
                                                             int budget) {
  const int nmesh = ctl->nmesh;
  int ndone = 0, apply = 0;
  for (int i0 = 0; i0 < nmesh; i0 += kBlock) {
    const int i = i0 + threadIdx.x;
    int d = 0, ap = 0;
    if (i < nmesh) {
      d = mds[i].s->done != 0;
      ap = !d && mds[i].s->phase == kPhaseApply;
    }
    ndone += __syncthreads_count(d);
    apply |= __syncthreads_or(ap);
  }
  if (threadIdx.x == 0) {
    ctl->cnt = 0u;
    ctl->iter = 0;
    ctl->cap = budget;
    ctl->all_done = ndone == nmesh ? 1 : 0;
    ctl->any_apply = apply;
    ctl->ndone_start = ndone;
  }
  rebuild_active(mds, ctl);
  if (apply && ctl->app_mesh) rebuild_apply(mds, ctl);
}

__global__ void collect_done_kernel(const MeshDev* __restrict__ mds, int nmesh, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nmesh) out[i] = mds[i].s->done;
}

}  // namespace

cudaError_t group_iterate(Group& g, int k, int mixed, int budget, int* done_host, cudaStream_t st) {
  loop_reset_kernel<<<1, kBlock, 0, st>>>(g.mds, g.ctl, budget);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (mixed) {
    e = group_host_loop_mixed(g, k, budget, st);
  } else {
    switch (k) {
      case 1: e = host_loop_k<1>(g, budget, 8, st); break;
      case 2: e = host_loop_k<2>(g, budget, 8, st); break;
      case 3: e = host_loop_k<3>(g, budget, 8, st); break;
      case 4: e = host_loop_k<4>(g, budget, 8, st); break;
      default: return cudaErrorInvalidValue;
    }
  }
  if (e != cudaSuccess) return e;
  if (!done_host) return cudaSuccess;
  if (!g.flags_dev) {
    e = cudaMalloc(&g.flags_dev, sizeof(int) * g.nmesh);
    if (e != cudaSuccess) return e;
  }
  collect_done_kernel<<<(g.nmesh + 255) / 256, 256, 0, st>>>(g.mds, g.nmesh, g.flags_dev);
  e = cudaMemcpyAsync(done_host, g.flags_dev, sizeof(int) * g.nmesh, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

cudaError_t group_begin(Group& g, int k, int mixed, const IoTable& io, int rhs_mass, const ig_solve_opts& o,
                        cudaStream_t st) {
  if (mixed) return group_begin_mixed(g, k, io, rhs_mass, o, st);
  switch (k) {
    case 1: return begin_k<1>(g, io, rhs_mass, o, st);
    case 2: return begin_k<2>(g, io, rhs_mass, o, st);
    case 3: return begin_k<3>(g, io, rhs_mass, o, st);
    case 4: return begin_k<4>(g, io, rhs_mass, o, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t group_end(Group& g, int k, const IoTable& io, cudaStream_t st) {
  switch (k) {
    case 1: return end_k<1>(g, io, st);
    case 2: return end_k<2>(g, io, st);
    case 3: return end_k<3>(g, io, st);
    case 4: return end_k<4>(g, io, st);
    default: return cudaErrorInvalidValue;
  }
}


int solver_blocks_per_sm() {
  int a = 0, b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, spmv_kernel<3>, kBlock, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, update_kernel<3>, kBlock, 0);
  const int m = a < b ? a : b;
  return m > 0 ? m : 1;
}

cudaError_t group_init(Group& g, const MeshDev* host_mds, int nmesh, int slots64, int slots32, cudaStream_t st) {
  g.nmesh = nmesh;
  g.host_mds.assign(host_mds, host_mds + nmesh);
  std::vector<int2> tiles, tiles32, ftiles, rtiles;
  for (int i = 0; i < nmesh; ++i) {
    for (int t = 0; t < host_mds[i].ntiles; ++t) tiles.push_back(make_int2(i, t));
    for (int t = 0; t < host_mds[i].ntiles32; ++t) tiles32.push_back(make_int2(i, t));
    for (int t = 0; t < (host_mds[i].m + 255) / 256; ++t) ftiles.push_back(make_int2(i, t));
    for (int t = 0; t < (host_mds[i].n + 255) / 256; ++t) rtiles.push_back(make_int2(i, t));
  }
  g.ntiles = (int)tiles.size();
  g.ntiles32 = (int)tiles32.size();
  g.grid64 = g.ntiles < slots64 ? g.ntiles : (slots64 > 0 ? slots64 : 1);
  g.grid32 = g.ntiles32 < slots32 ? g.ntiles32 : (slots32 > 0 ? slots32 : 1);
  if (g.grid32 < 1) g.grid32 = 1;
  g.nface_tiles = (int)ftiles.size();
  g.nrow_tiles = (int)rtiles.size();
  cudaError_t e;
  if ((e = cudaMalloc(&g.mds, sizeof(MeshDev) * nmesh)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&g.tiles, sizeof(int2) * tiles.size())) != cudaSuccess) return e;
  if ((e = cudaMalloc(&g.tiles32, sizeof(int2) * (tiles32.size() ? tiles32.size() : 1))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&g.face_tiles, sizeof(int2) * ftiles.size())) != cudaSuccess) return e;
  if ((e = cudaMalloc(&g.row_tiles, sizeof(int2) * rtiles.size())) != cudaSuccess) return e;
  if ((e = cudaMalloc(&g.ctl, sizeof(LoopCtl))) != cudaSuccess) return e;
  // ints: act_mesh, act_off64, act_off32, big_mesh, app_mesh, app_off32, app_big; then (16-byte
  // aligned) the int4 start tables start64, start32, app_start32
  const size_t list_ints = (7 * (size_t)nmesh + 3 + 3) / 4 * 4;
  const size_t list_words = list_ints + 4 * (size_t)(g.grid64 + 2 * g.grid32);
  if ((e = cudaMalloc(&g.act_buf, sizeof(int) * list_words)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&g.calls_dev, sizeof(CallDev) * nmesh)) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&g.calls_host, sizeof(CallDev) * nmesh)) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&g.done_host, sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaEventCreateWithFlags(&g.calls_ev, cudaEventDisableTiming)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(g.mds, host_mds, sizeof(MeshDev) * nmesh, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(g.tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return e;
  if (!tiles32.empty() && (e = cudaMemcpyAsync(g.tiles32, tiles32.data(), sizeof(int2) * tiles32.size(),
                                               cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(g.face_tiles, ftiles.data(), sizeof(int2) * ftiles.size(), cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(g.row_tiles, rtiles.data(), sizeof(int2) * rtiles.size(), cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return e;
  {
    LoopCtl c{};
    c.nmesh = nmesh;
    c.grid64 = g.grid64;
    c.grid32 = g.grid32;
    c.ndone_list = -1;
    int* w = g.act_buf;
    c.act_mesh = w;
    c.act_off64 = w + nmesh;
    c.act_off32 = w + 2 * (size_t)nmesh + 1;
    c.big_mesh = w + 3 * (size_t)nmesh + 2;
    c.app_mesh = w + 4 * (size_t)nmesh + 2;
    c.app_off32 = w + 5 * (size_t)nmesh + 2;
    c.app_big = w + 6 * (size_t)nmesh + 3;
    c.start64 = reinterpret_cast<int4*>(w + list_ints);
    c.start32 = c.start64 + g.grid64;
    c.app_start32 = c.start32 + g.grid32;
    g.list64 = ListRef{c.start64, c.act_mesh, c.big_mesh, &g.ctl->nbig};
    g.list32 = ListRef{c.start32, c.act_mesh, c.big_mesh, &g.ctl->nbig};
    g.listapp = ListRef{c.app_start32, c.app_mesh, c.app_big, &g.ctl->napp_big};
    if ((e = cudaMemcpyAsync(g.ctl, &c, sizeof(LoopCtl), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  }
  if ((e = cudaStreamCreateWithFlags(&g.capture_stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(g.calls_ev, st)) != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

// Refresh the device copy of the mesh descriptors from g.host_mds.
cudaError_t group_upload_mds(Group& g, cudaStream_t st) {
  return cudaMemcpyAsync(g.mds, g.host_mds.data(), sizeof(MeshDev) * g.nmesh, cudaMemcpyHostToDevice, st);
}

// Upload per-call arguments; waits until the previous upload from the pinned staging is done.
cudaError_t group_set_calls(Group& g, const CallDev* calls, cudaStream_t st) {
  cudaError_t e = cudaEventSynchronize(g.calls_ev);
  if (e != cudaSuccess) return e;
  std::memcpy(g.calls_host, calls, sizeof(CallDev) * g.nmesh);
  e = cudaMemcpyAsync(g.calls_dev, g.calls_host, sizeof(CallDev) * g.nmesh, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaEventRecord(g.calls_ev, st);
}

void group_destroy(Group& g) {
  for (auto& row : g.plans)
    for (auto& pl : row) {
      if (pl.exec) cudaGraphExecDestroy(pl.exec);
      if (pl.graph) cudaGraphDestroy(pl.graph);
      pl = SolvePlan{};
    }
  if (g.calls_ev) cudaEventSynchronize(g.calls_ev);
  if (g.capture_stream) cudaStreamDestroy(g.capture_stream);
  if (g.mds) cudaFree(g.mds);
  if (g.tiles) cudaFree(g.tiles);
  if (g.tiles32) cudaFree(g.tiles32);
  if (g.face_tiles) cudaFree(g.face_tiles);
  if (g.row_tiles) cudaFree(g.row_tiles);
  if (g.ctl) cudaFree(g.ctl);
  if (g.act_buf) cudaFree(g.act_buf);
  if (g.calls_dev) cudaFree(g.calls_dev);
  if (g.calls_host) cudaFreeHost(g.calls_host);
  if (g.done_host) cudaFreeHost(g.done_host);
  if (g.calls_ev) cudaEventDestroy(g.calls_ev);
  if (g.flags_dev) cudaFree(g.flags_dev);
  g = Group{};
}

cudaError_t group_solve(Group& g, int k, int mixed, const IoTable& io, int rhs_mass, const ig_solve_opts& o,
                        cudaStream_t st) {
  if (mixed) return group_solve_mixed(g, k, io, rhs_mass, o, st);
  switch (k) {
    case 1: return solve_k<1>(g, io, rhs_mass, o, st);
    case 2: return solve_k<2>(g, io, rhs_mass, o, st);
    case 3: return solve_k<3>(g, io, rhs_mass, o, st);
    case 4: return solve_k<4>(g, io, rhs_mass, o, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t group_true_residual(Group& g, int k, const IoTable& io, int rhs_mass, cudaStream_t st) {
  switch (k) {
    case 1: residual_kernel<1><<<g.ntiles, kBlock, 0, st>>>(g.mds, g.tiles, io, rhs_mass); break;
    case 2: residual_kernel<2><<<g.ntiles, kBlock, 0, st>>>(g.mds, g.tiles, io, rhs_mass); break;
    case 3: residual_kernel<3><<<g.ntiles, kBlock, 0, st>>>(g.mds, g.tiles, io, rhs_mass); break;
    case 4: residual_kernel<4><<<g.ntiles, kBlock, 0, st>>>(g.mds, g.tiles, io, rhs_mass); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace ig

// =============================================================================================
// Allocation-free solve on a caller-provided CSR operator.
//
// Some callers cannot allocate device memory at all: code that runs under a fixed memory plan
// or a pre-reserved arena (an embedded or real-time host that forbids cudaMalloc after start-up,
// a process whose allocator belongs to another framework), or code that must not add new
// allocations between two points of a stream. ig_solve_csr_noalloc serves them: it runs the same
// Jacobi-PCG kernels as ig_solve, with every piece of solver workspace (vectors, partial sums,
// loop state, the preconditioner) in one file-scope device array of fixed size, and the caller
// passes only inputs and outputs.
namespace ig {
namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr int kNoAllocMaxRows = IG_NOALLOC_MAX_ROWS;
constexpr int kNoAllocMaxTiles = (kNoAllocMaxRows + kTileRows - 1) / kTileRows;
constexpr size_t kNaMd = 0;
constexpr size_t kNaTiles = align256(kNaMd + sizeof(MeshDev));
constexpr size_t kNaCtl = align256(kNaTiles + sizeof(int2) * kNoAllocMaxTiles);
constexpr size_t kNaScal = align256(kNaCtl + sizeof(LoopCtl));
constexpr size_t kNaErr = align256(kNaScal + sizeof(SolveScal));
constexpr size_t kNaPart = align256(kNaErr + sizeof(int));
constexpr size_t kNaDinv = align256(kNaPart + sizeof(double) * kPartStride * kNoAllocMaxTiles);
constexpr size_t kNaVec = sizeof(double) * kMaxK * kNoAllocMaxRows;
constexpr size_t kNaX = align256(kNaDinv + sizeof(double) * kNoAllocMaxRows);
constexpr size_t kNaR = align256(kNaX + kNaVec);
constexpr size_t kNaP = align256(kNaR + kNaVec);
constexpr size_t kNaQ = align256(kNaP + kNaVec);
constexpr size_t kNaZ = align256(kNaQ + kNaVec);
constexpr size_t kNaList = align256(kNaZ + kNaVec);   // active lists of the one mesh: 8 ints
constexpr size_t kNaStart = align256(kNaList + sizeof(int) * 8);
constexpr size_t kNoAllocBytes = align256(kNaStart + sizeof(int4) * (kNoAllocMaxTiles + 1));

// Per-device base address of the scratch array, looked up once per device.
std::mutex g_noalloc_mu;
void* g_noalloc_base[64] = {};

// The caller's pattern checked (row ranges within [0, nnz), columns within [0, n)), the preconditioner
// from the operator's diagonal, solver state cleared, tile table written.
__global__ void __launch_bounds__(256) noalloc_setup_kernel(MeshDev md, MeshDev* md_out, int2* tiles, int ntiles,
                                                            LoopCtl ctl_init, LoopCtl* ctl, SolveScal* s) {
  const long row = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row < md.n) {
    double d = 0.0;
    const int e0 = md.rowptr[row], e1 = md.rowptr[row + 1];
    if (e0 < 0 || e1 < e0 || e1 > md.nnz) {
      atomicOr(md.err, kErrIndex);  // a row range outside the caller's [0, nnz)
    } else {
      for (int e = e0; e < e1; ++e) {
        const int c = md.col[e];
        if (c < 0 || c >= md.n) atomicOr(md.err, kErrIndex);  // a column outside [0, n)
        else if (c == row) d = md.A[e];
      }
    }
    if (!positive_finite(d)) atomicOr(md.err, kErrDegenerate);
    md.Dinv[row] = positive_finite(d) ? 1.0 / d : 0.0;
#pragma unroll
    for (int c = 0; c < kMaxK; ++c) md.p[row * kMaxK + c] = 0.0;
  }
  if (blockIdx.x == 0) {
    if (threadIdx.x < ntiles) tiles[threadIdx.x] = make_int2(0, threadIdx.x);
    if (threadIdx.x == 0) {
      *md_out = md;
      *ctl = ctl_init;
      *s = SolveScal{};
    }
  }
}

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

}  // namespace ig

extern "C" ig_status ig_solve_csr_noalloc(const int32_t* rowptr_dev, const int32_t* col_dev, const double* Aval_dev,
                                          const double* M_dev, int64_t n, int64_t nnz, const double* B_dev, int k,
                                          double* U_dev, void* cuda_stream, const ig_solve_opts* opts,
                                          ig_solve_info* info) {
  IG_NVTX("ig_solve_csr_noalloc");
  using namespace ig;
  if (!rowptr_dev || !col_dev || !Aval_dev || !B_dev || !U_dev) return IG_ERR_INVALID_ARG;
  if (n < 1 || n > kNoAllocMaxRows || nnz < n || nnz > (int64_t)INT32_MAX) return IG_ERR_INVALID_ARG;
  if (k < 1 || k > kMaxK || (const void*)B_dev == (const void*)U_dev) return IG_ERR_INVALID_ARG;
  ig_solve_opts o;
  ig_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.rel_tol >= 0.0) || !(o.rel_tol < 1e300) || o.max_iter < 1 || o.max_iter > 100000000)
    return IG_ERR_INVALID_ARG;
  o.launch = IG_LAUNCH_HOST;  // no graph objects are created on this path
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return IG_ERR_CUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return IG_ERR_CUDA;
      }
      g_noalloc_base[dev] = p;
    }
    base = static_cast<unsigned char*>(g_noalloc_base[dev]);
  }
  MeshDev md{};
  md.n = (int)n;
  md.nnz = (int)nnz;
  md.tile_rows = kTileRows;
  md.ntiles = (int)((n + kTileRows - 1) / kTileRows);
  md.k = k;
  md.rowptr = rowptr_dev;
  md.col = col_dev;
  md.A = const_cast<double*>(Aval_dev);
  md.M = const_cast<double*>(M_dev);
  md.Dinv = reinterpret_cast<double*>(base + kNaDinv);
  md.x = reinterpret_cast<double*>(base + kNaX);
  md.r = reinterpret_cast<double*>(base + kNaR);
  md.p = reinterpret_cast<double*>(base + kNaP);
  md.q = reinterpret_cast<double*>(base + kNaQ);
  md.z = reinterpret_cast<double*>(base + kNaZ);
  md.part = reinterpret_cast<double*>(base + kNaPart);
  md.s = reinterpret_cast<SolveScal*>(base + kNaScal);
  md.err = reinterpret_cast<int*>(base + kNaErr);
  Group g;
  g.nmesh = 1;
  g.ntiles = md.ntiles;
  {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return IG_ERR_CUDA;
    const int slots = sms * solver_blocks_per_sm();
    g.grid64 = md.ntiles < slots ? md.ntiles : slots;
  }
  g.mds = reinterpret_cast<MeshDev*>(base + kNaMd);
  g.tiles = reinterpret_cast<int2*>(base + kNaTiles);
  g.ctl = reinterpret_cast<LoopCtl*>(base + kNaCtl);
  int done_word = 0;
  g.done_host = &done_word;
  if (cudaMemsetAsync(md.err, 0, sizeof(int), st) != cudaSuccess) return IG_ERR_CUDA;
  LoopCtl ctl_init{};
  ctl_init.nmesh = 1;
  ctl_init.grid64 = g.grid64;
  ctl_init.grid32 = 0;
  ctl_init.ndone_list = -1;
  ctl_init.act_mesh = reinterpret_cast<int*>(base + kNaList);
  ctl_init.act_off64 = ctl_init.act_mesh + 1;
  ctl_init.act_off32 = ctl_init.act_mesh + 3;
  ctl_init.big_mesh = ctl_init.act_mesh + 5;
  ctl_init.start64 = reinterpret_cast<int4*>(base + kNaStart);
  ctl_init.start32 = ctl_init.start64 + kNoAllocMaxTiles;
  g.list64 = ListRef{ctl_init.start64, ctl_init.act_mesh, ctl_init.big_mesh,
                     &reinterpret_cast<LoopCtl*>(base + kNaCtl)->nbig};
  noalloc_setup_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(md, g.mds, g.tiles, g.ntiles, ctl_init, g.ctl, md.s);
  if (cudaGetLastError() != cudaSuccess) return IG_ERR_CUDA;
  // The caller's pattern is validated before the solve touches it: a row range outside [0, nnz)
  // or a column outside [0, n) would send the SpMV's loads out of the caller's arrays.
  {
    int bits0 = 0;
    if (cudaMemcpyAsync(&bits0, md.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return IG_ERR_CUDA;
    if (bits0) {
      const ig_status bad = (bits0 & kErrIndex) ? IG_ERR_INDEX_OUT_OF_RANGE : IG_ERR_INVALID_ARG;
      if (info) {
        std::memset(info, 0, sizeof(*info));
        info->status = bad;
        info->k = k;
      }
      return bad;
    }
  }
  // the pointer table lives on this thread's stack (16 KB): no host heap allocation either
  IoTable io;
  io.in[0] = B_dev;
  io.out[0] = U_dev;
  cudaError_t e = group_solve(g, k, 0, io, M_dev ? 1 : 0, o, st);
  if (e == cudaSuccess && info) e = group_true_residual(g, k, io, M_dev ? 1 : 0, st);
  if (e != cudaSuccess) return IG_ERR_CUDA;
  // The error word is always read back (the host loop has synchronised the stream already): a
  // missing or non-positive diagonal is a fault of the caller's operator, reported with or
  // without info.
  SolveScal s;
  int bits = 0;
  if ((info && cudaMemcpyAsync(&s, md.s, sizeof(SolveScal), cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
      cudaMemcpyAsync(&bits, md.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return IG_ERR_CUDA;
  if (!info) return bits ? IG_ERR_INVALID_ARG : IG_OK;
  std::memset(info, 0, sizeof(*info));
  info->status = bits ? IG_ERR_INVALID_ARG : s.status;
  info->k = k;
  info->iterations = s.iter;
  for (int c = 0; c < k; ++c) {
    info->rel_residual[c] = s.relres[c];
    info->true_rel_residual[c] = s.trueres[c];
  }
  return (ig_status)info->status;
}
