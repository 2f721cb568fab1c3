// ig_fairing.cu -- the element-wise steps of the inverse-fairing loop (§7.1): the M-norm loss
// 1/2 ||T - U||_M^2 = 1/2 sum_i M_i |T_i - U_i|^2 with its adjoint right-hand side and mass
// weights, and the preconditioned gradient step on the positions.
//
// One step (driven by ig_fairing_step in ig_api.cu, every piece on the device):
//   assemble A = M(V) + t L(V); U = A^-1 M V;
//   d = U - T, G = M d (dl/dU), w_i = |d_i|^2 / 2, loss = sum_i M_i w_i;
//   Lambda = A^-1 G; g = dl/dV = <Lambda, d(M V)/dV - (dA/dV) U> + d(sum_i M_i w_i)/dV;
//   Sobolev H^1 step: g~ = A^-1 g (the same operator: the gradient's Riesz representer in the
//   metric M + t L); V <- V - eta g~.
#include "ig_device.cuh"

namespace ig {

namespace {

// d = U - T, G = M d, w = |d|^2 / 2 per row; the loss sum_i M_i w_i reduced in tile order (the
// last CTA writes it to *loss). One CTA per FP64 solver tile of the (single) mesh.
__global__ void __launch_bounds__(kBlock) mnorm_kernel(const MeshDev* __restrict__ mds,
                                                       const int2* __restrict__ tiles,
                                                       const double* __restrict__ U,
                                                       const double* __restrict__ T, double* __restrict__ G,
                                                       double* __restrict__ w, double* __restrict__ loss) {
  __shared__ double sh[kBlock];
  const int2 tl = tiles[blockIdx.x];
  const MeshDev& md = mds[tl.x];
  const long nn = md.n;
  const long t0 = (long)tl.y * md.tile_rows;
  const long t1 = t0 + md.tile_rows < nn ? t0 + md.tile_rows : nn;
  double acc[1] = {0.0};
  for (long row = t0 + threadIdx.x; row < t1; row += kBlock) {
    const double m = md.M[row];
    double e = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double d = U[3 * row + c] - T[3 * row + c];
      G[3 * row + c] = m * d;
      e = fma(d, d, e);
    }
    w[row] = 0.5 * e;
    acc[0] = fma(m, 0.5 * e, acc[0]);
  }
  if (reduce_tiles<1>(acc, md.part, tl.y, md.ntiles, &md.s->cnt[2], sh) && threadIdx.x == 0) *loss = acc[0];
}

// V <- V - eta g over 3n values.
__global__ void __launch_bounds__(kBlock) step_kernel(double* __restrict__ V, const double* __restrict__ g,
                                                      double eta, long count) {
  for (long i = (long)blockIdx.x * kBlock + threadIdx.x; i < count; i += (long)gridDim.x * kBlock)
    V[i] = fma(-eta, g[i], V[i]);
}

}  // namespace

cudaError_t launch_mnorm(Group& g, const double* U, const double* T, double* G, double* w, double* loss,
                         cudaStream_t st) {
  IG_PROF("fair_mnorm", st);
  mnorm_kernel<<<g.ntiles, kBlock, 0, st>>>(g.mds, g.tiles, U, T, G, w, loss);
  return cudaGetLastError();
}

cudaError_t launch_step(double* V, const double* g, double eta, long count, int num_sms, cudaStream_t st) {
  IG_PROF("fair_step", st);
  long blocks = (count + kBlock - 1) / kBlock;
  const long cap = 4L * (num_sms > 0 ? num_sms : 1);
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  step_kernel<<<(int)blocks, kBlock, 0, st>>>(V, g, eta, count);
  return cudaGetLastError();
}

}  // namespace ig
