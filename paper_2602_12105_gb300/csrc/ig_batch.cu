// ig_batch.cu -- batches: many meshes assembled, solved and differentiated by the same kernel
// launches (block-diagonal system; every mesh keeps its own scalars, convergence and reductions).
//
// A batch is a launch group over meshes that were uploaded separately. Because each tile belongs
// to one mesh and each mesh's reductions add its own tile partials in tile order, a mesh gives
// the same bits alone and inside any batch.
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "ig_internal.cuh"

using namespace ig;

struct ig_batch {
  ig_ctx* ctx = nullptr;
  std::vector<ig_mesh*> meshes;
  Group group;
};

namespace {

ig_status batch_cuda(ig_ctx* ctx, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return IG_OK;
  set_error(ctx, std::string(where) + ": " + cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return IG_ERR_OOM;
  }
  return IG_ERR_CUDA;
}

#define BT_CK(ctx, call, where)                                     \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return batch_cuda((ctx), e_, (where));   \
  } while (0)

struct BatchDevice {
  int prev = -1;
  explicit BatchDevice(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~BatchDevice() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

ig_status bad(ig_ctx* ctx, const char* msg) {
  set_error(ctx, msg);
  return IG_ERR_INVALID_ARG;
}

// Refresh the batch's copy of the mesh descriptors (a mesh may have gained FP32 buffers).
cudaError_t refresh(ig_batch* b, cudaStream_t st) {
  for (size_t i = 0; i < b->meshes.size(); ++i) b->group.host_mds[i] = b->meshes[i]->md;
  return group_upload_mds(b->group, st);
}

ig_status batch_info(ig_batch* b, int k, ig_solve_info* infos) {
  ig_ctx* ctx = b->ctx;
  const size_t nm = b->meshes.size();
  std::vector<SolveScal> ss(nm);
  std::vector<int> bits(nm);
  for (size_t i = 0; i < nm; ++i) {
    BT_CK(ctx, cudaMemcpyAsync(&ss[i], b->meshes[i]->md.s, sizeof(SolveScal), cudaMemcpyDeviceToHost, ctx->stream),
          "read state");
    BT_CK(ctx, cudaMemcpyAsync(&bits[i], b->meshes[i]->md.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
          "read state");
  }
  BT_CK(ctx, cudaStreamSynchronize(ctx->stream), "batch solve");
  ig_status worst = IG_OK;
  for (size_t i = 0; i < nm; ++i) {
    ig_status st = (ig_status)ss[i].status;
    if (bits[i])
      st = (bits[i] & kErrBounds) ? IG_ERR_INDEX_OUT_OF_RANGE
                                  : ((bits[i] & kErrNonfinite) ? IG_ERR_NONFINITE : IG_ERR_DEGENERATE_FACE);
    if (st != IG_OK && worst == IG_OK) worst = st;
    if (infos) {
      ig_solve_info& inf = infos[i];
      std::memset(&inf, 0, sizeof(inf));
      inf.status = st;
      inf.k = k;
      inf.iterations = ss[i].iter;
      inf.refinements = ss[i].refine;
      for (int c = 0; c < k; ++c) {
        inf.rel_residual[c] = ss[i].relres[c];
        inf.true_rel_residual[c] = ss[i].trueres[c];
      }
    }
  }
  if (worst != IG_OK) set_error(ctx, "at least one mesh of the batch failed; see its ig_solve_info");
  return worst;
}

ig_solve_opts opts_or_default(const ig_solve_opts* o) {
  ig_solve_opts d;
  ig_default_opts(&d);
  return o ? *o : d;
}

}  // namespace

extern "C" {

ig_status ig_batch_create(ig_ctx* ctx, ig_mesh* const* meshes, int count, ig_batch** out) {
  IG_NVTX("ig_batch_create");
  if (!ctx || !out) return IG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!meshes || count < 1 || count > kMaxIo) return bad(ctx, "need 1 <= count <= 1024 meshes");
  for (int i = 0; i < count; ++i) {
    if (!meshes[i] || meshes[i]->ctx != ctx) return bad(ctx, "every mesh must belong to this context");
    for (int j = 0; j < i; ++j)
      if (meshes[j] == meshes[i]) return bad(ctx, "a mesh appears twice in the batch");
  }
  BatchDevice guard(ctx->device);
  std::unique_ptr<ig_batch> b(new (std::nothrow) ig_batch());
  if (!b) return IG_ERR_OOM;
  b->ctx = ctx;
  b->meshes.assign(meshes, meshes + count);
  std::vector<MeshDev> mds(count);
  for (int i = 0; i < count; ++i) mds[i] = meshes[i]->md;
  cudaError_t e = group_init(b->group, mds.data(), count, ctx->solver_slots, ctx->solver_slots32, ctx->stream);
  if (e != cudaSuccess) {
    group_destroy(b->group);
    return batch_cuda(ctx, e, "batch create");
  }
  ctx->live_meshes += 1;  // a live batch also keeps the context alive
  *out = b.release();
  return IG_OK;
}

ig_status ig_batch_free(ig_batch* b) {
  IG_NVTX("ig_batch_free");
  if (!b) return IG_ERR_INVALID_ARG;
  BatchDevice guard(b->ctx->device);
  cudaStreamSynchronize(b->ctx->stream);
  group_destroy(b->group);
  b->ctx->live_meshes -= 1;
  delete b;
  return IG_OK;
}

ig_status ig_batch_assemble(ig_batch* b, const double* const* V_dev, const double* t, int precision) {
  IG_NVTX("ig_batch_assemble");
  if (!b) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = b->ctx;
  if (!V_dev || !t) return bad(ctx, "V and t arrays are required");
  if (precision != IG_PRECISION_FP64 && precision != IG_PRECISION_MIXED && precision != IG_PRECISION_MIXED_GEOM32)
    return bad(ctx, "unknown precision");
  const int nm = (int)b->meshes.size();
  for (int i = 0; i < nm; ++i) {
    if (!V_dev[i]) return bad(ctx, "a V pointer is NULL");
    if (!(t[i] >= 0.0) || !std::isfinite(t[i])) return bad(ctx, "every t must be finite and >= 0");
  }
  BatchDevice guard(ctx->device);
  std::vector<CallDev> calls(nm);
  for (int i = 0; i < nm; ++i) {
    ig_mesh* m = b->meshes[i];
    if (precision == IG_PRECISION_MIXED) BT_CK(ctx, mesh_ensure_mixed(m, ctx->stream), "alloc");
    if (precision == IG_PRECISION_MIXED_GEOM32) BT_CK(ctx, mesh_ensure_geom32(m, ctx->stream), "alloc");
    BT_CK(ctx, mesh_set_geom32(m, precision == IG_PRECISION_MIXED_GEOM32 ? 1 : 0, ctx->stream), "upload");
    BT_CK(ctx, cudaMemsetAsync(m->md.err, 0, sizeof(int), ctx->stream), "memset");
    calls[i] = CallDev{};
    calls[i].V = V_dev[i];
    calls[i].t = t[i];
  }
  BT_CK(ctx, refresh(b, ctx->stream), "upload");
  BT_CK(ctx, group_set_calls(b->group, calls.data(), ctx->stream), "upload");
  BT_CK(ctx, launch_assemble(b->group, precision, ctx->stream), "batch assemble");
  for (int i = 0; i < nm; ++i) {
    b->meshes[i]->assembled = precision + 1;
    b->meshes[i]->t = t[i];
  }
  return IG_OK;
}

ig_status ig_batch_solve(ig_batch* b, const double* const* B_dev, int k, double* const* U_dev,
                         const ig_solve_opts* opts, ig_solve_info* infos) {
  IG_NVTX("ig_batch_solve");
  if (!b) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = b->ctx;
  const int nm = (int)b->meshes.size();
  if (!B_dev || !U_dev) return bad(ctx, "B and U arrays are required");
  if (k < 1 || k > kMaxK) return bad(ctx, "k must be in [1, 4]");
  const int prec = b->meshes[0]->assembled;
  for (int i = 0; i < nm; ++i) {
    if (!b->meshes[i]->assembled) {
      set_error(ctx, "batch solve before assemble");
      return IG_ERR_STATE;
    }
    if (b->meshes[i]->assembled != prec) return bad(ctx, "meshes of a batch must share one precision");
    if (!B_dev[i] || !U_dev[i] || (const void*)B_dev[i] == (const void*)U_dev[i])
      return bad(ctx, "B/U pointers must be non-NULL and distinct");
  }
  const ig_solve_opts o = opts_or_default(opts);
  if (!(o.rel_tol >= 0.0) || o.max_iter < 1 || o.max_refine < 1 || !(o.inner_tol > 0.0 && o.inner_tol < 1.0))
    return bad(ctx, "bad options");
  BatchDevice guard(ctx->device);
  auto io = std::make_unique<IoTable>();
  for (int i = 0; i < nm; ++i) {
    io->in[i] = B_dev[i];
    io->out[i] = U_dev[i];
  }
  BT_CK(ctx, refresh(b, ctx->stream), "upload");
  BT_CK(ctx, group_solve(b->group, k, prec >= 2, *io, 1, o, ctx->stream), "batch solve");
  if (!infos) return IG_OK;
  BT_CK(ctx, group_true_residual(b->group, k, *io, 1, ctx->stream), "residual");
  return batch_info(b, k, infos);
}

ig_status ig_batch_adjoint(ig_batch* b, const double* const* V_dev, const double* const* B_dev, int b_is_V,
                           const double* const* U_dev, const double* const* G_dev, int k, double* const* gV_dev,
                           double* const* gB_dev, double* gt_dev, const ig_solve_opts* opts,
                           ig_solve_info* infos) {
  IG_NVTX("ig_batch_adjoint");
  if (!b) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = b->ctx;
  const int nm = (int)b->meshes.size();
  if (!V_dev || !U_dev || !G_dev || !gV_dev) return bad(ctx, "V, U, G and gV arrays are required");
  if (!b_is_V && !B_dev) return bad(ctx, "B array required unless b_is_V");
  if (k < 1 || k > kMaxK || (b_is_V && k != 3)) return bad(ctx, "bad k");
  const int prec = b->meshes[0]->assembled;
  for (int i = 0; i < nm; ++i) {
    if (!b->meshes[i]->assembled) {
      set_error(ctx, "batch adjoint before assemble");
      return IG_ERR_STATE;
    }
    if (b->meshes[i]->assembled != prec) return bad(ctx, "meshes of a batch must share one precision");
    if (!V_dev[i] || !U_dev[i] || !G_dev[i] || !gV_dev[i] || (!b_is_V && !B_dev[i]))
      return bad(ctx, "a required pointer is NULL");
  }
  const ig_solve_opts o = opts_or_default(opts);
  if (!(o.rel_tol >= 0.0) || o.max_iter < 1 || o.max_refine < 1 || !(o.inner_tol > 0.0 && o.inner_tol < 1.0))
    return bad(ctx, "bad options");
  BatchDevice guard(ctx->device);
  auto io = std::make_unique<IoTable>();
  std::vector<CallDev> calls(nm);
  for (int i = 0; i < nm; ++i) {
    io->in[i] = G_dev[i];
    io->out[i] = b->meshes[i]->md.lam;
    CallDev& c = calls[i];
    c = CallDev{};
    c.V = V_dev[i];
    c.B = b_is_V ? V_dev[i] : B_dev[i];
    c.U = U_dev[i];
    c.gV = gV_dev[i];
    c.gB = gB_dev ? gB_dev[i] : nullptr;
    c.gt = gt_dev ? gt_dev + i : nullptr;
    c.t = b->meshes[i]->t;
    c.b_is_V = b_is_V ? 1 : 0;
    c.bstride = b_is_V ? 3 : k;
  }
  BT_CK(ctx, refresh(b, ctx->stream), "upload");
  BT_CK(ctx, group_solve(b->group, k, prec >= 2, *io, 0, o, ctx->stream), "batch adjoint solve");
  BT_CK(ctx, group_set_calls(b->group, calls.data(), ctx->stream), "upload");
  BT_CK(ctx, launch_vjp(b->group, k, ctx->stream, 0, prec == 3), "batch vjp");
  if (!infos) return IG_OK;
  BT_CK(ctx, group_true_residual(b->group, k, *io, 0, ctx->stream), "residual");
  return batch_info(b, k, infos);
}

ig_status ig_batch_iterate(ig_batch* b, int k, int max_iters, int* done_host) {
  IG_NVTX("ig_batch_iterate");
  if (!b) return IG_ERR_INVALID_ARG;
  ig_ctx* ctx = b->ctx;
  if (k < 1 || k > kMaxK) return bad(ctx, "k must be in [1, 4]");
  if (max_iters < 1) return bad(ctx, "max_iters must be >= 1");
  const int prec = b->meshes[0]->assembled;
  for (auto* m : b->meshes) {
    if (!m->assembled) {
      set_error(ctx, "iterate before assemble");
      return IG_ERR_STATE;
    }
    if (m->assembled != prec) return bad(ctx, "meshes of a batch must share one precision");
  }
  BatchDevice guard(ctx->device);
  BT_CK(ctx, refresh(b, ctx->stream), "upload");
  BT_CK(ctx, group_iterate(b->group, k, prec >= 2, max_iters, done_host, ctx->stream), "batch iterate");
  return IG_OK;
}

}  // extern "C"
