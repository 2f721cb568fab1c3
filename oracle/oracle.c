/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the implicit mesh-smoothing path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library calls, links or includes this
 * file; only the tests, the package's smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (the paper's inverse mean-curvature-flow step, §7.1, and the adjoint rule
 * for linear solves, §5.2 "Differentiating linear solvers", built on Eq. 3 of §3.1):
 *
 *   per face     : cotangent of each corner and the face area (the cotangent Laplacian L(v)
 *                  and the diagonal mass matrix M(v) of §7.1)
 *   operator     : A = M + t L, with L in the positive-semidefinite convention
 *                  (L_ab = -1/2 (cot alpha_ab + cot beta_ab), L_aa = -sum_b L_ab), so that
 *                  A equals the paper's M - tau L_paper with L_paper = -L
 *   forward      : A U = M B           (the paper's (M - tau L) v' = M v when B = V)
 *   adjoint      : A Lambda = G        (A is symmetric, so A^T = A)
 *   gradient     : dl/dtheta = <Lambda, d(M B)/dtheta - (dA/dtheta) U>
 *                  gathered per face in closed form (see orc_vjp)
 *
 * Every routine is the plain definition: a triplet list sorted into CSR, a dense Cholesky
 * factorisation or a textbook Jacobi-preconditioned conjugate gradient, and a face loop for
 * the gradient. No blocking, fusion or reordering beyond that.
 *
 * Readings where the paper is silent: barycentric lumping M_ii = sum over faces at i of
 * area/3; no cotangent clamp on this path unless asked for (the *_clamp variants: every
 * corner's cotangent clamped from below, the cotangent weights with a minimum of the paper's
 * §4 ARAP listing); a face with zero area is an error (status 3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_INDEX 2
#define ORC_ERR_DEGENERATE 3
#define ORC_ERR_NOT_CONVERGED 4
#define ORC_ERR_NONFINITE 5
#define ORC_ERR_OOM 6
#define ORC_ERR_NOT_SPD 8

/* ------------------------------------------------------------------------- small vectors */
static void sub3(const double* a, const double* b, double* o) {
  o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------- validation */
/* Every index in range, no repeated vertex in a face, every vertex used by some face. */
int orc_validate(int64_t n, int64_t m, const int32_t* F) {
  if (n <= 0 || m <= 0 || !F) return ORC_ERR_ARG;
  char* used = (char*)calloc((size_t)n, 1);
  if (!used) return ORC_ERR_OOM;
  int st = ORC_OK;
  for (int64_t f = 0; f < m && st == ORC_OK; ++f) {
    int32_t a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
    if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n) { st = ORC_ERR_INDEX; break; }
    if (a == b || b == c || a == c) { st = ORC_ERR_DEGENERATE; break; }
    used[a] = used[b] = used[c] = 1;
  }
  for (int64_t v = 0; v < n && st == ORC_OK; ++v)
    if (!used[v]) st = ORC_ERR_ARG;
  free(used);
  return st;
}

/* ------------------------------------------------------------------------- per-face geometry */
/* §7.1: L(v) is the cotangent Laplacian and M(v) the (diagonal) mass, both functions of the
 * positions. For face (i, j, k) with e_j = p_j - p_i, e_k = p_k - p_i and s = |e_j x e_k|:
 * area = s / 2 and cot of the angle at i = (e_j . e_k) / s; the other two corners cyclically.
 * cot is [m][3] (corner order of F), area is [m]. */
int orc_face_geometry(int64_t n, const double* V, int64_t m, const int32_t* F, double* cot, double* area) {
  (void)n;
  for (int64_t f = 0; f < m; ++f) {
    for (int c = 0; c < 3; ++c) {
      const double* pi = V + 3 * (int64_t)F[3 * f + c];
      const double* pj = V + 3 * (int64_t)F[3 * f + (c + 1) % 3];
      const double* pk = V + 3 * (int64_t)F[3 * f + (c + 2) % 3];
      double ej[3], ek[3], x[3];
      sub3(pj, pi, ej);
      sub3(pk, pi, ek);
      cross3(ej, ek, x);
      double s = sqrt(dot3(x, x));
      if (!(s > 0.0)) return ORC_ERR_DEGENERATE;
      cot[3 * f + c] = dot3(ej, ek) / s;
      if (c == 0) area[f] = 0.5 * s;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- Laplacian (CSR) */
typedef struct {
  int64_t row, col, seq;
  double val;
} orc_triplet;

static int triplet_cmp(const void* pa, const void* pb) {
  const orc_triplet* a = (const orc_triplet*)pa;
  const orc_triplet* b = (const orc_triplet*)pb;
  if (a->row != b->row) return a->row < b->row ? -1 : 1;
  if (a->col != b->col) return a->col < b->col ? -1 : 1;
  if (a->seq != b->seq) return a->seq < b->seq ? -1 : 1;
  return 0;
}

/* Cotangent Laplacian (PSD convention) as CSR. Each corner c of each face, with opposite
 * edge (a, b), adds w = cot_c / 2 as four triplets: (a,b) -w, (b,a) -w, (a,a) +w, (b,b) +w.
 * Triplets are sorted by (row, col, generation order) and equal keys are summed, so every
 * entry is summed in face order. rowptr has n+1 entries; col and val need capacity
 * cap >= n + 6m. With clamp non-NULL every corner's cotangent is first clamped from below,
 * cot_c <- max(cot_c, *clamp) (the cotangent weights with a minimum of the paper's §4 ARAP
 * listing, read per corner). Returns nnz (> 0) or minus an error code. */
static int64_t laplacian_csr(int64_t n, const double* V, int64_t m, const int32_t* F, const double* clamp,
                             int64_t* rowptr, int32_t* col, double* val, int64_t cap) {
  double* cot = (double*)malloc(sizeof(double) * 3 * (size_t)m);
  double* area = (double*)malloc(sizeof(double) * (size_t)m);
  orc_triplet* T = (orc_triplet*)malloc(sizeof(orc_triplet) * 12 * (size_t)m);
  if (!cot || !area || !T) { free(cot); free(area); free(T); return -ORC_ERR_OOM; }
  int st = orc_face_geometry(n, V, m, F, cot, area);
  if (st != ORC_OK) { free(cot); free(area); free(T); return -st; }
  int64_t nt = 0;
  for (int64_t f = 0; f < m; ++f) {
    for (int c = 0; c < 3; ++c) {
      int64_t a = F[3 * f + (c + 1) % 3], b = F[3 * f + (c + 2) % 3];
      double ct = cot[3 * f + c];
      if (clamp && ct < *clamp) ct = *clamp;
      double w = 0.5 * ct;
      orc_triplet t0 = {a, b, nt, -w}; T[nt++] = t0;
      orc_triplet t1 = {b, a, nt, -w}; T[nt++] = t1;
      orc_triplet t2 = {a, a, nt, w}; T[nt++] = t2;
      orc_triplet t3 = {b, b, nt, w}; T[nt++] = t3;
    }
  }
  qsort(T, (size_t)nt, sizeof(orc_triplet), triplet_cmp);
  int64_t nnz = 0;
  for (int64_t r = 0; r <= n; ++r) rowptr[r] = 0;
  for (int64_t i = 0; i < nt;) {
    int64_t j = i;
    double sum = 0.0;
    while (j < nt && T[j].row == T[i].row && T[j].col == T[i].col) { sum += T[j].val; ++j; }
    if (nnz >= cap) { free(cot); free(area); free(T); return -ORC_ERR_ARG; }
    col[nnz] = (int32_t)T[i].col;
    val[nnz] = sum;
    rowptr[T[i].row + 1] += 1;
    ++nnz;
    i = j;
  }
  for (int64_t r = 0; r < n; ++r) rowptr[r + 1] += rowptr[r];
  free(cot); free(area); free(T);
  return nnz;
}

int64_t orc_laplacian_csr(int64_t n, const double* V, int64_t m, const int32_t* F, int64_t* rowptr,
                          int32_t* col, double* val, int64_t cap) {
  return laplacian_csr(n, V, m, F, NULL, rowptr, col, val, cap);
}

/* The same with every corner's cotangent clamped from below at clamp_min. */
int64_t orc_laplacian_csr_clamp(int64_t n, const double* V, int64_t m, const int32_t* F, double clamp_min,
                                int64_t* rowptr, int32_t* col, double* val, int64_t cap) {
  return laplacian_csr(n, V, m, F, &clamp_min, rowptr, col, val, cap);
}

/* Barycentric lumped mass: M_ii = sum over faces containing i of area / 3 (face order). */
int orc_mass(int64_t n, const double* V, int64_t m, const int32_t* F, double* Mdiag) {
  double* cot = (double*)malloc(sizeof(double) * 3 * (size_t)m);
  double* area = (double*)malloc(sizeof(double) * (size_t)m);
  if (!cot || !area) { free(cot); free(area); return ORC_ERR_OOM; }
  int st = orc_face_geometry(n, V, m, F, cot, area);
  if (st == ORC_OK) {
    for (int64_t i = 0; i < n; ++i) Mdiag[i] = 0.0;
    for (int64_t f = 0; f < m; ++f)
      for (int c = 0; c < 3; ++c) Mdiag[F[3 * f + c]] += area[f] / 3.0;
  }
  free(cot); free(area);
  return st;
}

/* A = M + t L on the pattern of L (the pattern always holds the diagonal). */
int orc_operator(int64_t n, const int64_t* rowptr, const int32_t* col, const double* Lval, const double* Mdiag,
                 double t, double* Aval) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) Aval[e] = t * Lval[e] + (col[e] == i ? Mdiag[i] : 0.0);
  return ORC_OK;
}

/* Y = A X for X, Y of shape [n][k] (row-major). */
void orc_spmv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, int k, const double* X,
              double* Y) {
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < k; ++c) {
      double s = 0.0;
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += val[e] * X[(int64_t)col[e] * k + c];
      Y[i * k + c] = s;
    }
}

/* ------------------------------------------------------------------------- dense Cholesky */
/* Brute force for small n: densify A, factor A = L L^T (textbook column Cholesky), then
 * forward and back substitution for each of the k columns of R. X is [n][k]. */
int orc_dense_cholesky_solve(int64_t n, const int64_t* rowptr, const int32_t* col, const double* Aval, int k,
                             const double* R, double* X) {
  double* D = (double*)calloc((size_t)(n * n), sizeof(double));
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  if (!D || !y) { free(D); free(y); return ORC_ERR_OOM; }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) D[i * n + col[e]] += Aval[e];
  for (int64_t j = 0; j < n; ++j) {
    double d = D[j * n + j];
    for (int64_t p = 0; p < j; ++p) d -= D[j * n + p] * D[j * n + p];
    if (!(d > 0.0)) { free(D); free(y); return ORC_ERR_NOT_SPD; }
    double ljj = sqrt(d);
    D[j * n + j] = ljj;
    for (int64_t i = j + 1; i < n; ++i) {
      double s = D[i * n + j];
      for (int64_t p = 0; p < j; ++p) s -= D[i * n + p] * D[j * n + p];
      D[i * n + j] = s / ljj;
    }
  }
  for (int c = 0; c < k; ++c) {
    for (int64_t i = 0; i < n; ++i) {
      double s = R[i * k + c];
      for (int64_t p = 0; p < i; ++p) s -= D[i * n + p] * y[p];
      y[i] = s / D[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int64_t p = i + 1; p < n; ++p) s -= D[p * n + i] * X[p * k + c];
      X[i * k + c] = s / D[i * n + i];
    }
  }
  free(D); free(y);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- Jacobi-PCG */
/* Textbook preconditioned conjugate gradient with the Jacobi preconditioner diag(A)^-1,
 * one column of R at a time, x0 = 0, stopping when ||r||_2 / ||R_col||_2 <= tol (recursive
 * residual) or after max_iter iterations. iters[c] receives the iteration count and
 * relres[c] the TRUE relative residual ||R_col - A x||_2 / ||R_col||_2 recomputed at the end.
 * Returns ORC_ERR_NOT_CONVERGED if some column missed tol (its best iterate is still in X). */
int orc_pcg_solve(int64_t n, const int64_t* rowptr, const int32_t* col, const double* Aval, int k,
                  const double* R, double* X, double tol, int max_iter, int* iters, double* relres) {
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* z = (double*)malloc(sizeof(double) * (size_t)n);
  double* p = (double*)malloc(sizeof(double) * (size_t)n);
  double* q = (double*)malloc(sizeof(double) * (size_t)n);
  if (!d || !x || !r || !z || !p || !q) { free(d); free(x); free(r); free(z); free(p); free(q); return ORC_ERR_OOM; }
  int st = ORC_OK;
  for (int64_t i = 0; i < n; ++i) {
    d[i] = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (col[e] == i) d[i] = Aval[e];
    if (!(d[i] > 0.0)) st = ORC_ERR_NOT_SPD;
  }
  for (int c = 0; c < k && st != ORC_ERR_NOT_SPD; ++c) {
    double bn = 0.0;
    for (int64_t i = 0; i < n; ++i) { double b = R[i * k + c]; bn += b * b; }
    bn = sqrt(bn);
    double rz = 0.0, rr = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      x[i] = 0.0;
      r[i] = R[i * k + c];
      z[i] = r[i] / d[i];
      p[i] = z[i];
      rz += r[i] * z[i];
      rr += r[i] * r[i];
    }
    int it = 0;
    while (bn > 0.0 && sqrt(rr) / bn > tol && it < max_iter) {
      for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += Aval[e] * p[col[e]];
        q[i] = s;
      }
      double pq = 0.0;
      for (int64_t i = 0; i < n; ++i) pq += p[i] * q[i];
      if (!(pq > 0.0) || !isfinite(pq)) { st = ORC_ERR_NONFINITE; break; }
      double alpha = rz / pq;
      double rz_new = 0.0;
      rr = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
        z[i] = r[i] / d[i];
        rz_new += r[i] * z[i];
        rr += r[i] * r[i];
      }
      double beta = rz_new / rz;
      rz = rz_new;
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
      ++it;
    }
    /* true residual */
    double tr = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += Aval[e] * x[col[e]];
      double ri = R[i * k + c] - s;
      tr += ri * ri;
      X[i * k + c] = x[i];
    }
    if (iters) iters[c] = it;
    double rel = bn > 0.0 ? sqrt(tr) / bn : 0.0;
    if (relres) relres[c] = rel;
    if (st == ORC_OK && bn > 0.0 && sqrt(rr) / bn > tol) st = ORC_ERR_NOT_CONVERGED;
  }
  free(d); free(x); free(r); free(z); free(p); free(q);
  return st;
}

/* ------------------------------------------------------------------------- gradient */
/* Adjoint rule for A(v) U = M(v) B (Eq. 3 of §3.1 with the linear-solve partials of §5.2):
 * with Lambda = A^-1 G,  dl/dtheta = <Lambda, d(M B)/dtheta - (dA/dtheta) U>, where <.,.>
 * sums over all rows and the k columns. With A = M + t L this splits per face f:
 *
 *   mass part : (d area_f / 3) * sum_{v in f} <Lambda_v, B_v - U_v>
 *   cot part  : -t * sum_{corners c} (1/2) d cot_c * <Lambda_a - Lambda_b, U_a - U_b>,
 *               (a, b) the edge opposite c
 *
 * using, for corner i of CCW face (i, j, k), e_j = p_j - p_i, e_k = p_k - p_i, s = |e_j x e_k|,
 * n = (e_j x e_k) / s:
 *   grad_{p_i} area = 1/2 n x (p_k - p_j)
 *   d cot_i / d e_j = (e_k - cot_i (e_k x n)) / s,   d cot_i / d e_k = (e_j - cot_i (n x e_j)) / s,
 *   d cot_i / d p_i = -(d cot_i / d e_j + d cot_i / d e_k).
 * When B is V itself (b_is_V), M Lambda is added to gV (the explicit dependence of M V on V).
 * Other outputs: gB = M Lambda (when B is independent of V; may be NULL) and
 * gt = -<Lambda, L U> (may be NULL). U, Lam, B are [n][k]; gV is [n][3]. */
/* With clamp non-NULL the operator was assembled from the clamped cotangents max(cot_c, *clamp):
 * a clamped corner (cot_c < *clamp) holds a constant, so it adds nothing to dl/dV, and dl/dt
 * uses the clamped value. */
static int vjp(int64_t n, const double* V, int64_t m, const int32_t* F, double t, int k, const double* U,
               const double* Lam, const double* B, int b_is_V, const double* clamp, double* gV, double* gB,
               double* gt) {
  if (b_is_V && k != 3) return ORC_ERR_ARG;
  const double* Bsrc = b_is_V ? V : B;
  double* M = (double*)calloc((size_t)n, sizeof(double));
  if (!M) return ORC_ERR_OOM;
  for (int64_t i = 0; i < 3 * n; ++i) gV[i] = 0.0;
  double gt_acc = 0.0;
  for (int64_t f = 0; f < m; ++f) {
    int64_t vid[3] = {F[3 * f], F[3 * f + 1], F[3 * f + 2]};
    const double* P[3] = {V + 3 * vid[0], V + 3 * vid[1], V + 3 * vid[2]};
    double e1[3], e2[3], x[3], nrm[3];
    sub3(P[1], P[0], e1);
    sub3(P[2], P[0], e2);
    cross3(e1, e2, x);
    double s = sqrt(dot3(x, x));
    if (!(s > 0.0)) { free(M); return ORC_ERR_DEGENERATE; }
    for (int d = 0; d < 3; ++d) nrm[d] = x[d] / s;
    double area = 0.5 * s;
    for (int a = 0; a < 3; ++a) M[vid[a]] += area / 3.0;

    /* mass part */
    double wa = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < k; ++c)
        wa += Lam[vid[a] * k + c] * (Bsrc[vid[a] * k + c] - U[vid[a] * k + c]);
    wa /= 3.0;
    for (int a = 0; a < 3; ++a) {
      double opp[3], g[3];
      sub3(P[(a + 2) % 3], P[(a + 1) % 3], opp);
      cross3(nrm, opp, g);
      for (int d = 0; d < 3; ++d) gV[vid[a] * 3 + d] += wa * 0.5 * g[d];
    }

    /* cotangent part */
    for (int ci = 0; ci < 3; ++ci) {
      int cj = (ci + 1) % 3, ck = (ci + 2) % 3;
      double ej[3], ek[3];
      sub3(P[cj], P[ci], ej);
      sub3(P[ck], P[ci], ek);
      double cot = dot3(ej, ek) / s;
      double lu = 0.0;
      for (int c = 0; c < k; ++c)
        lu += (Lam[vid[cj] * k + c] - Lam[vid[ck] * k + c]) * (U[vid[cj] * k + c] - U[vid[ck] * k + c]);
      if (clamp && cot < *clamp) {
        gt_acc -= 0.5 * (*clamp) * lu;
        continue;
      }
      gt_acc -= 0.5 * cot * lu;
      double w = -t * 0.5 * lu;
      double ekxn[3], nxej[3], dj[3], dk[3];
      cross3(ek, nrm, ekxn);
      cross3(nrm, ej, nxej);
      for (int d = 0; d < 3; ++d) {
        dj[d] = (ek[d] - cot * ekxn[d]) / s;
        dk[d] = (ej[d] - cot * nxej[d]) / s;
      }
      for (int d = 0; d < 3; ++d) {
        gV[vid[cj] * 3 + d] += w * dj[d];
        gV[vid[ck] * 3 + d] += w * dk[d];
        gV[vid[ci] * 3 + d] -= w * (dj[d] + dk[d]);
      }
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    for (int c = 0; c < k; ++c) {
      double ml = M[i] * Lam[i * k + c];
      if (gB) gB[i * k + c] = ml;
      if (b_is_V) gV[i * 3 + c] += ml;
    }
  }
  if (gt) *gt = gt_acc;
  free(M);
  return ORC_OK;
}

int orc_vjp(int64_t n, const double* V, int64_t m, const int32_t* F, double t, int k, const double* U,
            const double* Lam, const double* B, int b_is_V, double* gV, double* gB, double* gt) {
  return vjp(n, V, m, F, t, k, U, Lam, B, b_is_V, NULL, gV, gB, gt);
}

/* The gradient of the step assembled with clamped cotangents (orc_laplacian_csr_clamp). */
int orc_vjp_clamp(int64_t n, const double* V, int64_t m, const int32_t* F, double t, int k, const double* U,
                  const double* Lam, const double* B, int b_is_V, double clamp_min, double* gV, double* gB,
                  double* gt) {
  return vjp(n, V, m, F, t, k, U, Lam, B, b_is_V, &clamp_min, gV, gB, gt);
}

/* Gradient of the mass term sum_i M_i(v) w_i (M_i = sum over the faces at i of area/3) with
 * respect to the positions: for each face, ((1/3) sum_{v in f} w_v) times grad area_f, with
 * grad_{p_i} area = 1/2 n x (p_k - p_j) for CCW (i, j, k). This is how the M-norm objective
 * 1/2 ||t - g(v)||_M^2 of the inverse-fairing problem (§7.1) depends on v through M, with
 * w = |t - g(v)|^2 / 2. gV is [n][3] (overwritten). */
int orc_mass_vjp(int64_t n, const double* V, int64_t m, const int32_t* F, const double* w, double* gV) {
  for (int64_t i = 0; i < 3 * n; ++i) gV[i] = 0.0;
  for (int64_t f = 0; f < m; ++f) {
    int64_t vid[3] = {F[3 * f], F[3 * f + 1], F[3 * f + 2]};
    const double* P[3] = {V + 3 * vid[0], V + 3 * vid[1], V + 3 * vid[2]};
    double e1[3], e2[3], x[3], nrm[3];
    sub3(P[1], P[0], e1);
    sub3(P[2], P[0], e2);
    cross3(e1, e2, x);
    double s = sqrt(dot3(x, x));
    if (!(s > 0.0)) return ORC_ERR_DEGENERATE;
    for (int d = 0; d < 3; ++d) nrm[d] = x[d] / s;
    double wf = (w[vid[0]] + w[vid[1]] + w[vid[2]]) / 3.0;
    for (int a = 0; a < 3; ++a) {
      double opp[3], g[3];
      sub3(P[(a + 2) % 3], P[(a + 1) % 3], opp);
      cross3(nrm, opp, g);
      for (int d = 0; d < 3; ++d) gV[vid[a] * 3 + d] += wf * 0.5 * g[d];
    }
  }
  return ORC_OK;
}

/* Number of threads this oracle uses (it is single-threaded). */
int orc_num_threads(void) { return 1; }
