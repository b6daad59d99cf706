// Riemannian CG on products of generalized Stiefel manifolds with the
// preconditioned metric g(xi, eta) = tr(xi^T M eta), M = R^T R (Sec. 3, Table 1),
// for the CCA cost (Sec. 4.2) and the FDA cost (Sec. 5.2); warm start from the
// exact solution of the sketched problem (Alg. 1 step 4, Alg. 2 step 5); final
// Rayleigh-Ritz step.
//
// One iteration = one fused data pass at Phi = [U, eta] plus small kernels:
//   line search   every Gram the retraction and the cost need along
//                 t -> R_U(t eta) is a quadratic in t of k x k blocks of the
//                 pass Gram, so all trial steps are evaluated from the pass
//                 (35 trials in parallel, then the sequential Armijo rule);
//   update        U+ = (U + t eta) L^{-T} (QR retraction in Cholesky form,
//                 Table 1), B U+ and the Euclidean gradient from the linear
//                 pass outputs Z^T W (Sec. 4.2 gradient), no second pass;
//   M^{-1}        two products with R^{-1};
//   direction     one k x k eigendecomposition per factor solves the three
//                 Sylvester equations of the projection (Table 1) for the
//                 gradient and the two transported vectors; Hestenes-Stiefel
//                 beta (clipped at 0) in the metric g; restart if not descent;
//   new direction eta+ = -grad + beta T(eta), with its M-image carried along
//                 so no product with M is ever formed.
// Each kernel returns at once when the device flag `done` is set, so the host
// enqueues iterations in batches and reads the flag between batches.
#include "plan.h"

namespace gbcca {

constexpr double kC1 = 1e-4;
constexpr int kMaxLS = 25;
constexpr int kMaxExpand = 10;
constexpr int kNTrials = kMaxLS + kMaxExpand + 1;  // last one: t = 0 (Armijo reference)

// ================================================================ helpers
// Block-wide small dense routines on shared memory (row-major, FP64).
__device__ void blk_sync() { __syncthreads(); }

// C (m x n) = op(A) op(B), inner dimension q; C must not alias A or B.
__device__ void blk_mm(const double* A, bool tA, const double* B, bool tB, double* C, int m, int q, int n, int lda,
                       int ldb) {
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
    int i = e / n, j = e % n;
    double s = 0;
    for (int l = 0; l < q; ++l) s += (tA ? A[l * lda + i] : A[i * lda + l]) * (tB ? B[j * ldb + l] : B[l * ldb + j]);
    C[e] = s;
  }
  __syncthreads();
}

// Symmetric eigendecomposition by parallel (round-robin ordered) Jacobi:
// A (n x n, destroyed) -> eigenvalues in lam (descending), eigenvectors in
// the columns of Q (n x n).  rot is shared scratch of 3 * 33 doubles/ints.
template <typename R>
__device__ void blk_jacobi(R* A, R* Q, R* lam, int n, double* rot) {
  R* cs = reinterpret_cast<R*>(rot);
  R* sn = cs + 33;
  int* pp = reinterpret_cast<int*>(rot + 66);
  int* qq = pp + 33;
  __shared__ double offn;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) Q[e] = (e / n == e % n) ? 1.0 : 0.0;
  __syncthreads();
  const int m = n + (n & 1);
  __shared__ double s_off[32], s_dg[32];
  for (int sweep = 0; sweep < 20 && n > 1; ++sweep) {
    {
      R off = 0, dg = 0;
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        R v = A[e] * A[e];
        if (e / n == e % n) dg += v;
        else off += v;
      }
      off = warp_sum(off);
      dg = warp_sum(dg);
      if ((threadIdx.x & 31) == 0) {
        s_off[threadIdx.x >> 5] = off;
        s_dg[threadIdx.x >> 5] = dg;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double o = 0, d = 0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) {
          o += s_off[w];
          d += s_dg[w];
        }
        // off-diagonal norm below 1e-13 of the diagonal: the next sweep would
        // only move entries at the rounding level
        offn = (o <= (sizeof(R) == 8 ? 1e-26 : 1e-12) * d || o == 0.0) ? 1.0 : 0.0;
      }
      __syncthreads();
    }
    if (offn > 0.5) break;
    for (int r = 0; r < m - 1; ++r) {
      if (threadIdx.x < m / 2) {
        int i = threadIdx.x;
        int a = (i == 0) ? 0 : 1 + ((i - 1 + r) % (m - 1));
        int b = 1 + ((m - 2 - i + r) % (m - 1));
        int p = min(a, b), q = max(a, b);
        R c = 1, s = 0;
        if (q < n) {
          R apq = A[p * n + q];
          // rotations of entries far below the rounding level of the pivots are skipped
          const R eps = R(sizeof(R) == 8 ? 1e-17 : 1e-8);
          if (apq * apq > eps * eps * fabs(A[p * n + p] * A[q * n + q])) {
            R tau = (A[q * n + q] - A[p * n + p]) / (R(2) * apq);
            R t = (tau >= 0 ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
            c = R(1) / sqrt(R(1) + t * t);
            s = t * c;
          }
        }
        cs[i] = c;
        sn[i] = s;
        pp[i] = p;
        qq[i] = q < n ? q : -1;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = threadIdx.x; e < (m / 2) * n; e += blockDim.x) {
        int i = e / n, j = e % n;
        if (qq[i] < 0) continue;
        int p = pp[i], q = qq[i];
        R ap = A[p * n + j], aq = A[q * n + j];
        A[p * n + j] = cs[i] * ap - sn[i] * aq;
        A[q * n + j] = sn[i] * ap + cs[i] * aq;
      }
      __syncthreads();
      // columns: A <- A J, Q <- Q J
      for (int e = threadIdx.x; e < (m / 2) * n; e += blockDim.x) {
        int i = e / n, j = e % n;
        if (qq[i] < 0) continue;
        int p = pp[i], q = qq[i];
        R ap = A[j * n + p], aq = A[j * n + q];
        A[j * n + p] = cs[i] * ap - sn[i] * aq;
        A[j * n + q] = sn[i] * ap + cs[i] * aq;
        R qp = Q[j * n + p], qv = Q[j * n + q];
        Q[j * n + p] = cs[i] * qp - sn[i] * qv;
        Q[j * n + q] = sn[i] * qp + cs[i] * qv;
      }
      __syncthreads();
    }
  }
  // sort descending (selection sort by one thread, swapping Q columns)
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
    for (int i = 0; i < n; ++i) {
      int b = i;
      for (int j = i + 1; j < n; ++j)
        if (lam[j] > lam[b]) b = j;
      if (b != i) {
        R t = lam[i];
        lam[i] = lam[b];
        lam[b] = t;
        for (int r = 0; r < n; ++r) {
          R u = Q[r * n + i];
          Q[r * n + i] = Q[r * n + b];
          Q[r * n + b] = u;
        }
      }
    }
  }
  __syncthreads();
}

// The same parallel Jacobi sweeps for n <= 40 by one warp: rotation pairs
// on lanes, warp-level barriers only (the block version spends most of its
// time in block-wide barriers for matrices this small).  Called by all 32
// lanes of one warp.
template <typename R>
__device__ void warp_jacobi(R* A, R* Q, R* lam, int n, int max_sweeps = 20, R tol = R(0)) {
  if (!(tol > R(0))) tol = R(sizeof(R) == 8 ? 1e-26 : 1e-12);
  const int lane = threadIdx.x & 31;
  // rotation tables of this warp (up to 8 warps of a CTA may run their own
  // decompositions side by side)
  // (n <= 40: at most 20 rotations per round)
  __shared__ R w_cs_all[8][20], w_sn_all[8][20];
  __shared__ int w_p_all[8][20], w_q_all[8][20], w_rank_all[8][20];
  const int wslot = (threadIdx.x >> 5) & 7;
  R* w_cs = w_cs_all[wslot];
  R* w_sn = w_sn_all[wslot];
  int* w_p = w_p_all[wslot];
  int* w_q = w_q_all[wslot];
  for (int e = lane; e < n * n; e += 32) Q[e] = (e / n == e % n) ? R(1) : R(0);
  __syncwarp();
  const int m = n + (n & 1);
  R prev_off = R(-1);
  for (int sweep = 0; sweep < max_sweeps && n > 1; ++sweep) {
    R off = 0, dg = 0;
    for (int e = lane; e < n * n; e += 32) {
      const R v = A[e] * A[e];
      if (e / n == e % n) dg += v;
      else off += v;
    }
    off = warp_sum(off);
    dg = warp_sum(dg);
    if (off <= tol * dg || off == R(0)) break;
    // cyclic Jacobi converges quadratically: a sweep that no longer halves
    // the off-diagonal mass has reached the rounding floor of R
    if (prev_off >= R(0) && off > R(0.5) * prev_off) break;
    prev_off = off;
    for (int r = 0; r < m - 1; ++r) {
      if (lane < m / 2) {
        const int i = lane;
        const int a = (i == 0) ? 0 : 1 + ((i - 1 + r) % (m - 1));
        const int b = 1 + ((m - 2 - i + r) % (m - 1));
        const int p = min(a, b), q = max(a, b);
        R c = 1, sv = 0;
        if (q < n) {
          const R apq = A[p * n + q];
          const R eps = R(sizeof(R) == 8 ? 1e-17 : 1e-8);
          if (apq * apq > eps * eps * fabs(A[p * n + p] * A[q * n + q])) {
            const R tau = (A[q * n + q] - A[p * n + p]) / (R(2) * apq);
            const R t = (tau >= 0 ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
            c = R(1) / sqrt(R(1) + t * t);
            sv = t * c;
          }
        }
        w_cs[i] = c;
        w_sn[i] = sv;
        w_p[i] = p;
        w_q[i] = q < n ? q : -1;
      }
      __syncwarp();
      for (int e = lane; e < (m / 2) * n; e += 32) {  // rows: A <- J^T A
        const int i = e / n, j = e % n;
        if (w_q[i] < 0) continue;
        const int p = w_p[i], q = w_q[i];
        const R ap = A[p * n + j], aq = A[q * n + j];
        A[p * n + j] = w_cs[i] * ap - w_sn[i] * aq;
        A[q * n + j] = w_sn[i] * ap + w_cs[i] * aq;
      }
      __syncwarp();
      for (int e = lane; e < (m / 2) * n; e += 32) {  // columns: A <- A J, Q <- Q J
        const int i = e / n, j = e % n;
        if (w_q[i] < 0) continue;
        const int p = w_p[i], q = w_q[i];
        const R ap = A[j * n + p], aq = A[j * n + q];
        A[j * n + p] = w_cs[i] * ap - w_sn[i] * aq;
        A[j * n + q] = w_sn[i] * ap + w_cs[i] * aq;
        const R qp = Q[j * n + p], qv = Q[j * n + q];
        Q[j * n + p] = w_cs[i] * qp - w_sn[i] * qv;
        Q[j * n + q] = w_sn[i] * qp + w_cs[i] * qv;
      }
      __syncwarp();
    }
  }
  // sort descending (ties keep the lower index first)
  if (n <= 20) {
    // lane i < n finds the position of eigenvalue i, then the lanes move
    // the columns of Q there
    int* w_rank = w_rank_all[wslot];
    const R lv = lane < n ? A[lane * n + lane] : R(0);
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const R lj = __shfl_sync(0xffffffffu, lv, j);
      if (lj > lv || (lj == lv && j < lane)) ++rank;
    }
    if (lane < n) w_rank[lane] = rank;
    constexpr int kPer = (20 * 20 + 31) / 32;  // entries of Q per lane
    R qv[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = lane + 32 * u;
      qv[u] = e < n * n ? Q[e] : R(0);
    }
    __syncwarp();
    if (lane < n) lam[rank] = lv;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = lane + 32 * u;
      if (e < n * n) Q[(e / n) * n + w_rank[e % n]] = qv[u];
    }
  } else if (lane == 0) {  // selection sort, swapping Q columns
    for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
    for (int i = 0; i < n; ++i) {
      int b = i;
      for (int j = i + 1; j < n; ++j)
        if (lam[j] > lam[b]) b = j;
      if (b != i) {
        const R t = lam[i];
        lam[i] = lam[b];
        lam[b] = t;
        for (int rr = 0; rr < n; ++rr) {
          const R u = Q[rr * n + i];
          Q[rr * n + i] = Q[rr * n + b];
          Q[rr * n + b] = u;
        }
      }
    }
  }
  __syncwarp();
}

// In-place Cholesky A = L L^T (lower; upper part zeroed).  Returns false
// (uniformly in the block) if a pivot is not positive.
__device__ bool blk_chol(double* A, int n) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double dj = A[j * n + j];
      if (!(dj > 0.0)) {
        bad = 1;
        dj = 1.0;
      }
      A[j * n + j] = sqrt(dj);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * n + j] /= A[j * n + j];
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int i = e / n, c = e % n;
      if (i > j && c > j && c <= i) A[i * n + c] -= A[i * n + j] * A[c * n + j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x)
    if (e % n > e / n) A[e] = 0.0;
  __syncthreads();
  return bad == 0;
}

// Li = L^{-1} for lower-triangular L (n x n), column-parallel forward substitution.
__device__ void blk_lower_inv(const double* L, double* Li, int n) {
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    for (int i = 0; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int q = c; q < i; ++q) s -= L[i * n + q] * Li[q * n + c];
      Li[i * n + c] = (i < c) ? 0.0 : s / L[i * n + i];
    }
  }
  __syncthreads();
}

// Warp-level versions used by the parallel line-search trials (n <= 32).
// The reciprocal of each pivot is kept on the diagonal's mirror (invd) so the
// triangular solves multiply instead of divide.
__device__ bool warp_chol(double* A, int n, double* invd) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int j = 0; j < n; ++j) {
    double dj = A[j * n + j];
    if (!(dj > 0.0)) {
      ok = false;
      dj = 1.0;
    }
    const double rj = rsqrt_nr(dj);
    const double ljj = dj * rj;
    __syncwarp();
    if (lane == j) {
      A[j * n + j] = ljj;
      invd[j] = rj;
    }
    if (lane > j && lane < n) A[lane * n + j] *= rj;
    __syncwarp();
    // trailing update, one element (r, c), j < c <= r < n, per lane: FP64
    // instructions are slow to issue on this GPU, so as few warp-wide ones
    // as possible (the triangle of m rows has m (m + 1) / 2 elements)
    const int m = n - j - 1;
    for (int e = lane; e < m * (m + 1) / 2; e += 32) {
      int r = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);  // e = r (r + 1) / 2 + c'
      if ((r + 1) * (r + 2) / 2 <= e) ++r;
      if (r * (r + 1) / 2 > e) --r;
      const int rr = j + 1 + r, cc = j + 1 + (e - r * (r + 1) / 2);
      A[rr * n + cc] -= A[rr * n + j] * A[cc * n + j];
    }
    __syncwarp();
  }
  return ok;
}

// Li = L^{-1} (lane c computes column c)
__device__ void warp_lower_inv(const double* L, const double* invd, double* Li, int n) {
  const int c = threadIdx.x & 31;
  if (c < n) {
    for (int i = 0; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int q = c; q < i; ++q) s -= L[i * n + q] * Li[q * n + c];
      Li[i * n + c] = (i < c) ? 0.0 : s * invd[i];
    }
  }
  __syncwarp();
}

// ========================================================= thin Grams
// part[view][blk] (ca x cb) = A[rows of blk]^T B[rows of blk], A: d x ca
// (row stride lda), B: d x cb (ldb), kThinRows rows per block.
constexpr int kThinRows = 16;
struct ThinArgs {
  const double* A[2];
  const double* B[2];
  int lda[2], ldb[2], d[2];
  int ca, cb, nblk;
  double* part;
  const int* done;
};

__global__ void thin_gram_kernel(ThinArgs a) {
  extern __shared__ double tsm[];
  if (a.done != nullptr && *a.done) return;
  const int v = blockIdx.y;
  const int d = a.d[v];
  const int r0 = blockIdx.x * kThinRows;
  double* As = tsm;
  double* Bs = tsm + kThinRows * a.ca;
  const int nr = min(kThinRows, d - r0);
  for (int e = threadIdx.x; e < kThinRows * a.ca; e += blockDim.x) {
    int r = e / a.ca, c = e % a.ca;
    As[e] = r < nr ? a.A[v][(int64_t)(r0 + r) * a.lda[v] + c] : 0.0;
  }
  for (int e = threadIdx.x; e < kThinRows * a.cb; e += blockDim.x) {
    int r = e / a.cb, c = e % a.cb;
    Bs[e] = r < nr ? a.B[v][(int64_t)(r0 + r) * a.ldb[v] + c] : 0.0;
  }
  __syncthreads();
  double* out = a.part + ((int64_t)v * a.nblk + blockIdx.x) * a.ca * a.cb;
  for (int e = threadIdx.x; e < a.ca * a.cb; e += blockDim.x) {
    int i = e / a.cb, j = e % a.cb;
    double s = 0;
    for (int r = 0; r < nr; ++r) s += As[r * a.ca + i] * Bs[r * a.cb + j];
    out[e] = s;
  }
}

// out[v][e] = sum over row blocks b of part[v][b][e]: one warp per output,
// lanes over blocks, a fixed shuffle tree (deterministic), FP64.
__global__ void reduce_blocks_kernel(const double* __restrict__ part, int nblk, int len, int nviews,
                                     double* __restrict__ out, const int* done) {
  if (done != nullptr && *done) return;
  const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (gw >= nviews * len) return;
  const int v = gw / len, e = gw - v * len;
  const double* pv = part + (int64_t)v * nblk * len + e;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += pv[(int64_t)b * len];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[gw] = s;
}

static int thin_gram(Plan& p, const double* A0, const double* A1, int lda, const double* B0, const double* B1,
                     int ldb, int ca, int cb, double* part, cudaStream_t st, const int* done,
                     double* out = nullptr) {
  ThinArgs a{};
  a.A[0] = A0;
  a.A[1] = A1;
  a.B[0] = B0;
  a.B[1] = B1;
  int dmax = 0;
  for (int v = 0; v < p.nviews; ++v) {
    a.lda[v] = lda;
    a.ldb[v] = ldb;
    a.d[v] = p.v[v].d;
    dmax = std::max(dmax, p.v[v].d);
  }
  a.ca = ca;
  a.cb = cb;
  a.nblk = ceil_div(dmax, kThinRows);
  a.part = part;
  a.done = done;
  size_t smem = sizeof(double) * kThinRows * (ca + cb);
  GB_CUDA(cudaFuncSetAttribute(thin_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // blocks past a view's rows write zeros (nr <= 0 loops are empty)
  thin_gram_kernel<<<dim3(a.nblk, p.nviews), 256, smem, st>>>(a);
  GB_CHECK_LAUNCH();
  if (out != nullptr) {
    // partials summed by many CTAs, so the single-CTA consumers read one block
    const int64_t warps = (int64_t)p.nviews * ca * cb;
    reduce_blocks_kernel<<<ceil_div(warps * 32, 256), 256, 0, st>>>(part, a.nblk, ca * cb, p.nviews, out, done);
    GB_CHECK_LAUNCH();
  }
  return GBCCA_OK;
}

__device__ void sum_blocks(const double* part, int nblk, int len, double* out) {
  if (nblk == 1) {  // already summed: a copy (no FP64 additions of zeros), 8 loads in flight
    for (int e0 = threadIdx.x; e0 < len; e0 += 8 * blockDim.x) {
      double t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x;
        t[u] = e < len ? part[e] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < len) out[e] = t[u];
      }
    }
    __syncthreads();
    return;
  }
  // loads are issued 8 at a time (independent), then added in block order
  for (int e = threadIdx.x; e < len; e += blockDim.x) {
    double s = 0;
    for (int b0 = 0; b0 < nblk; b0 += 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (b0 + u < nblk) ? part[(int64_t)(b0 + u) * len + e] : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    out[e] = s;
  }
  __syncthreads();
}

// ============================================================ line search
struct LSArgs {
  DevState* st;
  const double* Gram;     // pass Gram (NC x NC)
  const double* phipart;  // [view][nblk][2k x 2k]
  int nblk;
  int NC, k, nviews, kind;
  const double* YPhi;     // FDA: Yhat Phi (l x 2k)
  int l;
  double* history;
  int max_iter;
  double* ls_f;           // kNTrials trial values
  double* ls_L;           // kNTrials x 2 x kMaxK^2 trial factors
  int polar;              // 1: polar retraction (factors Gram(t)^{-1/2})
};

// Work area of one line-search trial (doubles): Gram_x, Gram_y, Cross, two
// factors, two eigenvector matrices, one product (kk each), two k-vectors.
constexpr int ls_work_doubles(int k) { return 8 * k * k + 2 * kMaxK; }

// F = A^{-1/2} for a symmetric positive definite A (n x n, destroyed), by one
// warp: A = Q diag(w) Q^T by Jacobi rotations, F = Q diag(w^{-1/2}) Q^T.
// Returns false (on every lane) if an eigenvalue is not positive.
__device__ bool warp_inv_sqrt(double* A, double* Q, double* w, double* F, int n) {
  warp_jacobi<double>(A, Q, w, n);
  const int lane = threadIdx.x & 31;
  const bool ok = w[n - 1] > 0.0;  // eigenvalues sorted descending
  if (lane < n) w[lane] = ok ? 1.0 / sqrt(w[lane]) : 0.0;
  __syncwarp();
  for (int e = lane; e < n * n; e += 32) {
    const int r = e / n, c = e - r * n;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += Q[r * n + i] * w[i] * Q[c * n + i];
    F[e] = s;
  }
  __syncwarp();
  return ok;
}

// f(t) for one trial, evaluated by one warp from the coefficient matrices.
// coef layout per view v (k x k each): A_v, B_v, C_v  (Gram(t) = A + t B + t^2 C)
// and the cross / S_B terms X0, X1, X2 (Cross(t) = X0 + t X1 + t^2 X2).
__device__ double ls_eval(const LSArgs& a, const double* coef, double t, double* w, const double* mu) {
  const int k = a.k, kk = k * k, lane = threadIdx.x & 31;
  double* Gx = w;
  double* Gy = w + kk;
  double* Cx = w + 2 * kk;
  double* Li = w + 3 * kk;
  double* ix = w + 4 * kk;
  double* iy = ix + kMaxK;
  for (int e = lane; e < kk; e += 32) {
    Gx[e] = coef[e] + t * coef[kk + e] + t * t * coef[2 * kk + e];
    if (a.kind == kCCA) Gy[e] = coef[3 * kk + e] + t * coef[4 * kk + e] + t * t * coef[5 * kk + e];
    Cx[e] = coef[6 * kk + e] + t * coef[7 * kk + e] + t * t * coef[8 * kk + e];
  }
  __syncwarp();
  bool ok = warp_chol(Gx, k, ix);
  if (a.kind == kCCA) ok = warp_chol(Gy, k, iy) && ok;
  // Y = Lx^{-1} Cross  (lane c solves column c)
  if (lane < k) {
    for (int i = 0; i < k; ++i) {
      double s = Cx[i * k + lane];
      for (int q = 0; q < i; ++q) s -= Gx[i * k + q] * Cx[q * k + lane];
      Cx[i * k + lane] = s * ix[i];
    }
  }
  __syncwarp();
  // second factor: Ly (CCA) or Lx again (FDA: L^{-1} S_B L^{-T})
  if (a.kind == kCCA) warp_lower_inv(Gy, iy, Li, k);
  else warp_lower_inv(Gx, ix, Li, k);
  double part = 0;
  if (lane < k) {
    double z = 0;
    for (int j = 0; j <= lane; ++j) z += Cx[lane * k + j] * Li[lane * k + j];
    part = mu[lane] * z;
  }
  double f = -warp_sum(part);
  if (a.kind == kLDA) f *= 0.5;
  if (!ok || !(f == f)) f = INFINITY;
  return f;
}

// CCA trial by three warps of the CTA (called by all threads): warp 0
// factors Gx(t), warp 1 factors Gy(t) and inverts L_y at the same time (GB300
// issues FP64 slowly on each scheduler, so the two chains run side by side);
// then warp 0 forms f(t) while warp 2 inverts L_x for the stored factors.
// w: Gx, Gy, Cx, Ly^{-1}, Lx^{-1} (kk each), ix, iy (kMaxK each).
__device__ double ls_eval_cca_cta(const LSArgs& a, const double* coef, double t, double* w, const double* mu) {
  const int k = a.k, kk = k * k, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  double* Gx = w;
  double* Gy = w + kk;
  double* Cx = w + 2 * kk;
  double* Li = w + 3 * kk;
  double* Lt = w + 4 * kk;
  double* ix = w + 5 * kk;
  double* iy = ix + kMaxK;
  __shared__ int s_ok[2];
  __shared__ double s_f;
  for (int e = tid; e < kk; e += blockDim.x) {
    Gx[e] = coef[e] + t * coef[kk + e] + t * t * coef[2 * kk + e];
    Gy[e] = coef[3 * kk + e] + t * coef[4 * kk + e] + t * t * coef[5 * kk + e];
    Cx[e] = coef[6 * kk + e] + t * coef[7 * kk + e] + t * t * coef[8 * kk + e];
  }
  __syncthreads();
  if (warp == 0) {
    const bool ok = warp_chol(Gx, k, ix);
    if (lane == 0) s_ok[0] = ok;
  } else if (warp == 1) {
    const bool ok = warp_chol(Gy, k, iy);
    if (lane == 0) s_ok[1] = ok;
    warp_lower_inv(Gy, iy, Li, k);
  }
  __syncthreads();
  if (warp == 0) {
    // Y = Lx^{-1} Cross (lane c solves column c); f = -tr(N Y Ly^{-T})
    if (lane < k) {
      for (int i = 0; i < k; ++i) {
        double sv = Cx[i * k + lane];
        for (int q = 0; q < i; ++q) sv -= Gx[i * k + q] * Cx[q * k + lane];
        Cx[i * k + lane] = sv * ix[i];
      }
    }
    __syncwarp();
    double part = 0;
    if (lane < k) {
      double z = 0;
      for (int j = 0; j <= lane; ++j) z += Cx[lane * k + j] * Li[lane * k + j];
      part = mu[lane] * z;
    }
    double f = -warp_sum(part);
    if (!(s_ok[0] && s_ok[1]) || !(f == f)) f = INFINITY;
    if (lane == 0) s_f = f;
  } else if (warp == 2) {
    warp_lower_inv(Gx, ix, Lt, k);
  }
  __syncthreads();
  return s_f;
}

// Polar-retraction trial (called by all threads): warps 0 and 1 form
// F_x = Gram_x(t)^{-1/2} and F_y = Gram_y(t)^{-1/2} side by side (FDA: warp 0
// F = Gram(t)^{-1/2} only); the cost is f = -tr(N F_x Cross(t) F_y) (FDA:
// -1/2 tr(N F S_B(t) F)).  F_y (FDA: F) is left at w + 3kk and F_x at w + 4kk,
// where the Cholesky evaluators leave L_y^{-1} and L_x^{-1}: both factors are
// symmetric, so the transposed copy the caller makes is the factor itself.
__device__ double ls_eval_polar(const LSArgs& a, const double* coef, double t, double* w, const double* mu) {
  const int k = a.k, kk = k * k, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool cca = a.kind == kCCA;
  double* Gx = w;
  double* Gy = w + kk;
  double* Cx = w + 2 * kk;
  double* Fy = w + 3 * kk;
  double* Fx = cca ? w + 4 * kk : Fy;
  double* Qx = w + 5 * kk;
  double* Qy = w + 6 * kk;
  double* T = w + 7 * kk;
  double* ex = w + 8 * kk;
  double* ey = ex + kMaxK;
  __shared__ int s_okp[2];
  __shared__ double s_fp;
  for (int e = tid; e < kk; e += blockDim.x) {
    Gx[e] = coef[e] + t * coef[kk + e] + t * t * coef[2 * kk + e];
    if (cca) Gy[e] = coef[3 * kk + e] + t * coef[4 * kk + e] + t * t * coef[5 * kk + e];
    Cx[e] = coef[6 * kk + e] + t * coef[7 * kk + e] + t * t * coef[8 * kk + e];
  }
  if (tid == 0) s_okp[1] = 1;
  __syncthreads();
  if (warp == 0) {
    const bool ok = warp_inv_sqrt(Gx, Qx, ex, Fx, k);
    if (lane == 0) s_okp[0] = ok;
  } else if (warp == 1 && cca) {
    const bool ok = warp_inv_sqrt(Gy, Qy, ey, Fy, k);
    if (lane == 0) s_okp[1] = ok;
  }
  __syncthreads();
  for (int e = tid; e < kk; e += blockDim.x) {  // T = F_x Cross
    const int r = e / k, c = e - r * k;
    double sv = 0.0;
    for (int q = 0; q < k; ++q) sv += Fx[r * k + q] * Cx[q * k + c];
    T[e] = sv;
  }
  __syncthreads();
  if (warp == 0) {
    double part = 0.0;
    if (lane < k) {
      double z = 0.0;
      for (int j = 0; j < k; ++j) z += T[lane * k + j] * Fy[j * k + lane];
      part = mu[lane] * z;
    }
    double f = -warp_sum(part);
    if (!cca) f *= 0.5;
    if (!(s_okp[0] && s_okp[1]) || !(f == f)) f = INFINITY;
    if (lane == 0) s_fp = f;
  }
  __syncthreads();
  return s_fp;
}

// Every trial step of the sequential Armijo rule is evaluated at once, one
// CTA (one warp) per trial, so the FP64 work of the k x k Cholesky factors
// is spread over kNTrials SMs instead of queueing on one SM's FP64 pipe:
//   trial 0: t = 0 (the Armijo reference, at the point of this pass),
//   trials 1 .. kMaxExpand + 1: t0 2^0 .. t0 2^kMaxExpand (t0 and its expansions),
//   trials kMaxExpand + 2 ..: t0 2^-1 .. t0 2^-(kMaxLS - 1) (backtracking).
// Each CTA stores f(t) and the factors L_v(t)^{-T} of its trial; the last CTA
// to finish applies the sequential rule (first accepted backtracking step; or
// t0 and then doublings while f decreases and Armijo holds) to the stored
// values, so the accepted step is exactly the one of the sequential search.
__device__ __forceinline__ double ls_trial_t(int i, double t0) {
  if (i == 0) return 0.0;
  if (i <= kMaxExpand + 1) return ldexp(t0, i - 1);
  return ldexp(t0, -(i - kMaxExpand - 1));
}

__global__ void linesearch_kernel(LSArgs a) {
  DevState* st = a.st;
  if (st->done) return;
  extern __shared__ double lsm[];
  const int k = a.k, kk = k * k, k2 = 2 * k;
  const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
  const bool zero_step = st->force_zero_step != 0;
  double* coef = lsm;                       // 9 kk
  double* phig = coef + 9 * kk;             // 2 views x 4 kk
  double* w = phig + 8 * kk;                // ls_work_doubles(k)
  __shared__ double mu_s[kMaxK];
  __shared__ int last;
  if (!zero_step || i == 0) {
    // the whole CTA loads (several loads in flight per thread); warp 0 then
    // evaluates the trial
    if (tid < k) mu_s[tid] = st->mu[tid];
    for (int e = tid; e < a.nviews * 4 * kk; e += blockDim.x) phig[e] = a.phipart[e];
    __syncthreads();
    // coefficient matrices: Gram_v(t) = A + t B + t^2 C, Cross(t) = X0 + t X1 + t^2 X2
    const int NC = a.NC;
    for (int e = tid; e < kk; e += blockDim.x) {
      const int r = e / k, c = e % k;
      auto G = [&](int bi, int bj) { return a.Gram[(bi * k + r) * NC + bj * k + c]; };
      for (int v = 0; v < a.nviews; ++v) {
        const double* pg = phig + v * 4 * kk;  // 2k x 2k
        auto P = [&](int bi, int bj) { return pg[(bi * k + r) * k2 + bj * k + c]; };
        const double lam = st->lam[v];
        const int b0 = 2 * v;  // pass blocks of this view: [P_U, P_eta] or [Q_V, Q_eta]
        coef[(3 * v + 0) * kk + e] = G(b0, b0) + lam * P(0, 0);
        coef[(3 * v + 1) * kk + e] = G(b0, b0 + 1) + G(b0 + 1, b0) + lam * (P(0, 1) + P(1, 0));
        coef[(3 * v + 2) * kk + e] = G(b0 + 1, b0 + 1) + lam * P(1, 1);
      }
      if (a.kind == kCCA) {
        coef[6 * kk + e] = G(0, 2);
        coef[7 * kk + e] = G(0, 3) + G(1, 2);
        coef[8 * kk + e] = G(1, 3);
      } else {
        // S_B(t) = (Yhat W + t Yhat eta)^T (Yhat W + t Yhat eta)
        double s0 = 0, s1 = 0, s2 = 0;
        for (int cl = 0; cl < a.l; ++cl) {
          const double wi = a.YPhi[cl * k2 + r], wj = a.YPhi[cl * k2 + c];
          const double ei = a.YPhi[cl * k2 + k + r], ej = a.YPhi[cl * k2 + k + c];
          s0 += wi * wj;
          s1 += wi * ej + ei * wj;
          s2 += ei * ej;
        }
        coef[6 * kk + e] = s0;
        coef[7 * kk + e] = s1;
        coef[8 * kk + e] = s2;
      }
    }
    __syncthreads();
    const double t = ls_trial_t(i, st->t0);
    // factors L_v(t)^{-T} of this trial (row-major), kept for the decision
    double* Lout = a.ls_L + (int64_t)i * 2 * kMaxK * kMaxK;
    if (a.polar) {
      const double f = ls_eval_polar(a, coef, t, w, mu_s);
      const double* Fy = w + 3 * kk;
      const double* Fx = a.kind == kCCA ? w + 4 * kk : Fy;
      for (int e = tid; e < kk; e += blockDim.x) {
        Lout[e] = Fx[e];
        Lout[kMaxK * kMaxK + e] = Fy[e];
      }
      if (tid == 0) a.ls_f[i] = f;
    } else if (a.kind == kCCA) {
      const double f = ls_eval_cca_cta(a, coef, t, w, mu_s);
      const double* Li = w + 3 * kk;
      const double* Lt = w + 4 * kk;
      for (int e = tid; e < kk; e += blockDim.x) {
        const int r = e / k, c = e % k;
        Lout[e] = Lt[c * k + r];
        Lout[kMaxK * kMaxK + e] = Li[c * k + r];
      }
      if (tid == 0) a.ls_f[i] = f;
    } else if (tid < 32) {
      const double f = ls_eval(a, coef, t, w, mu_s);
      const double* Li = w + 3 * kk;
      for (int e = lane; e < kk; e += 32) {
        const int r = e / k, c = e % k;
        Lout[e] = Li[c * k + r];
      }
      if (lane == 0) a.ls_f[i] = f;
    }
  }
  // the last CTA to finish decides (warp 0 of it)
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(&st->ls_count, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!last || tid >= 32) return;
  __threadfence();
  if (lane == 0) st->ls_count = 0;
  // every trial value at once from L2 (two per lane; the other CTAs' stores
  // are visible there after their fences and atomics), then the sequential
  // rule on warp shuffles: all lanes take the same decisions
  static_assert(kNTrials <= 64, "two trial values per lane");
  const double fva = lane < (int)gridDim.x ? __ldcg(&a.ls_f[lane]) : 0.0;
  const double fvb = lane + 32 < (int)gridDim.x ? __ldcg(&a.ls_f[lane + 32]) : 0.0;
  auto fv = [&](int e) {
    const double x = __shfl_sync(0xffffffffu, fva, e & 31);
    const double y = __shfl_sync(0xffffffffu, fvb, e & 31);
    return e < 32 ? x : y;
  };
  const double t0 = st->t0, df = st->df;
  const double f0 = fv(0);
  int acc = -1, trials = 1;
  if (zero_step) {
    acc = 0;
  } else if (fv(1) <= f0 + kC1 * t0 * df) {
    acc = 1;
    trials = 2;
    for (int e = 2; e <= kMaxExpand + 1; ++e) {
      const double te = ls_trial_t(e, t0);
      ++trials;
      const double fe = fv(e);
      if (fe < fv(acc) && fe <= f0 + kC1 * te * df)
        acc = e;
      else
        break;
    }
  } else {
    trials = 2;
    for (int e = kMaxExpand + 2; e < (int)gridDim.x; ++e) {
      ++trials;
      if (fv(e) <= f0 + kC1 * ls_trial_t(e, t0) * df) {
        acc = e;
        break;
      }
    }
  }
  if (acc < 0) {
    if (lane == 0) {
      st->stalled = 1;
      st->done = 1;
      st->ls_trials = trials;
    }
    return;
  }
  const double t = ls_trial_t(acc, t0);
  const volatile double* L = a.ls_L + (int64_t)acc * 2 * kMaxK * kMaxK;
  for (int e = lane; e < kk; e += 32) {
    st->Linv[0][e] = L[e];
    if (a.kind == kCCA) st->Linv[1][e] = L[kMaxK * kMaxK + e];
  }
  __syncwarp();
  if (a.kind == kLDA) {
    // YW+ = (Yhat W + t Yhat eta) L^{-T}
    for (int e = lane; e < a.l * k; e += 32) {
      const int cl = e / k, c = e % k;
      double s = 0;
      for (int q = 0; q < k; ++q) s += (a.YPhi[cl * k2 + q] + t * a.YPhi[cl * k2 + k + q]) * st->Linv[0][q * k + c];
      st->YW[e] = s;
    }
  }
  const double f_acc = fv(acc);  // (all lanes: a shuffle)
  if (lane == 0) {
    st->t = t;
    st->f = f_acc;
    st->ls_trials = trials;
    if (!zero_step) {
      st->t_prev = t;
      st->df_prev = st->df;
      st->iter += 1;
    }
  }
}

// ================================================================ update
struct UpdArgs {
  DevState* st;
  const double* G;      // D x NC pass output
  int NC, k, nviews, kind, l, D;
  double* Phi[2];
  double* LL[2];
  double* RR[2];
  float* RRh[2];        // optional float-pair copy of RR[:, 0:2k]
  float* RRl[2];
  const double* Meta[2];
  const double* gold[2];
  const double* Mgold[2];
  int d[2];
  int dofs[2];
  const double* Yhat;   // FDA (l x d)
};

// View v, rows of this CTA: U+ = (U + t eta) Lv^{-T}; B U+; Euclidean
// gradient.  k threads per row (thread c of a row owns column c): the row
// vectors u_t = U + t eta, B-image and cross term are formed once per row in
// shared memory, then each thread forms its column of the three products.
// The CTA covers whole rows, so U can be overwritten after a barrier.
__global__ void update_kernel(UpdArgs a) {
  DevState* st = a.st;
  if (st->done) return;
  extern __shared__ double usm[];  // rows x 3k
  const int k = a.k, k2 = 2 * k, k4 = 4 * k;
  const int rows = blockDim.x / k;
  const int v = blockIdx.y;
  const int lr = threadIdx.x / k, c = threadIdx.x - lr * k;
  const int j = blockIdx.x * rows + lr;
  const bool act = lr < rows && j < a.d[v];
  const double t = st->t, lam = st->lam[v];
  double* Phi = a.Phi[v] + (int64_t)j * k2;
  double* ut = usm + lr * 3 * k;
  double* bt = ut + k;
  double* ct = bt + k;
  if (act) {
    // columns of W are [P_U, P_eta, Q_V, Q_eta]: own block gives the
    // B-image, the other block (CCA) the cross term
    const double* Grow = a.G + (int64_t)(a.dofs[v] + j) * a.NC;
    const int own = 2 * v, oth = 2 * (1 - v);
    const double u = Phi[c] + t * Phi[k + c];
    ut[c] = u;
    bt[c] = Grow[own * k + c] + t * Grow[(own + 1) * k + c] + lam * u;
    if (a.kind == kCCA) ct[c] = Grow[oth * k + c] + t * Grow[(oth + 1) * k + c];
  }
  __syncthreads();
  if (!act) return;
  const double* Li = st->Linv[v];
  double u = 0, b = 0, g = 0;
  for (int q = 0; q < k; ++q) {
    u += ut[q] * Li[q * k + c];
    b += bt[q] * Li[q * k + c];
  }
  if (a.kind == kCCA) {
    const double* Lo = st->Linv[1 - v];
    for (int q = 0; q < k; ++q) g += ct[q] * Lo[q * k + c];
  } else {
    // egrad = -S_B W+ N = -Yhat^T (Yhat W+) N
    for (int cl = 0; cl < a.l; ++cl) g += a.Yhat[(int64_t)cl * a.d[0] + j] * st->YW[cl * k + c];
  }
  g = -g * st->mu[c];
  double* LLr = a.LL[v] + (int64_t)j * k4;
  double* RRr = a.RR[v] + (int64_t)j * k4;
  // old direction and gradient (and their M-images) move to the Gram buffers
  LLr[2 * k + c] = Phi[k + c];
  LLr[3 * k + c] = a.gold[v][(int64_t)j * k + c];
  RRr[2 * k + c] = a.Meta[v][(int64_t)j * k + c];
  RRr[3 * k + c] = a.Mgold[v][(int64_t)j * k + c];
  Phi[c] = u;  // every thread of this row has read U (barrier above)
  RRr[c] = b;
  RRr[k + c] = g;
  if (a.RRh[v] != nullptr) {
    const float bh = (float)b, gh = (float)g;
    a.RRh[v][(int64_t)j * k2 + c] = bh;
    a.RRl[v][(int64_t)j * k2 + c] = (float)(b - (double)bh);
    a.RRh[v][(int64_t)j * k2 + k + c] = gh;
    a.RRl[v][(int64_t)j * k2 + k + c] = (float)(g - (double)gh);
  }
}

// ============================================================= direction
struct DirArgs {
  DevState* st;
  const double* crosspart;  // [view][nblk][4k x 4k]
  int nblk, k, nviews;
  double* history;
  int max_iter;
};

// Block-wide sum of NV per-thread values (blockDim a multiple of 32, <= 256):
// a shuffle tree per warp, then the warps' sums added in warp order
// (deterministic).
template <int NV>
__device__ void blk_sum(double (&v)[NV], double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0)
    for (int q = 0; q < NV; ++q) red[q * 8 + w] = v[q];
  __syncthreads();
  // the warps' sums added once, in warp order, by thread q (FP64 issue is
  // scarce: all threads repeating them cost more than the rest together)
  if (threadIdx.x < NV) {
    double t = 0;
    for (int i = 0; i < nw; ++i) t += red[threadIdx.x * 8 + i];
    red[NV * 8 + threadIdx.x] = t;
  }
  __syncthreads();
  for (int q = 0; q < NV; ++q) v[q] = red[NV * 8 + q];
  __syncthreads();
}

// Per factor: X = [Wn, xi, eta, g]^T [BU, egrad, M eta, M g] (4k x 4k blocks
// X[a][b]).  The projection of Table 1 needs S with A S + S A = C + C^T for
// A = sym(X[0][0]) = U^T B M^{-1} B U and C = X[a][0]^T (a = 1: gradient,
// 2: old direction, 3: old gradient); A = Q diag(lam) Q^T gives
// S = Q ((Q^T (C + C^T) Q) ./ (lam_i + lam_j)) Q^T.  Inner products in g of
// u = L_a - Wn Su with M w = R_b - BU Sw expand into
//   tr X[a][b] - tr(X[a][0] Sw) - tr(Su^T X[0][b]) + tr(Su^T X[0][0] Sw).
template <typename R>
__global__ void direction_kernel(DirArgs a) {
  DevState* st = a.st;
  if (st->done) return;
  extern __shared__ double dsm[];
  const int k = a.k, kk = k * k, k4 = 4 * k;
  double* X = dsm;                 // 16 kk per view (FP64 cross Gram)
  double* Y = X + 2 * 16 * kk;     // 2 kk: X00 Sg, X00 So (FP64), then 3 kk: S (FP64)
  double* rot = Y + 5 * kk;        // 100
  double* red = rot + 100;         // 6 x 256
  R* A = reinterpret_cast<R*>(red + 6 * 256);  // kk
  R* Q = A + kk;                   // kk
  R* lam = Q + kk;                 // kMaxK
  R* T = lam + kMaxK;              // 3 kk
  R* T2 = T + 3 * kk;              // 3 kk
  R* S = T2 + 3 * kk;              // 3 kk (this view's S_g, S_e, S_o)
  // one CTA per view; the last CTA to finish combines the views' sums
  const int v = blockIdx.x;
  sum_blocks(a.crosspart + (int64_t)v * a.nblk * 16 * kk, a.nblk, 16 * kk, X + v * 16 * kk);
  double acc[6] = {0, 0, 0, 0, 0, 0};  // gg, g_Tg, Te_g, Te_Tg, dfg, dfTe
  {
    const double* Xv = X + v * 16 * kk;
    auto XB = [&](int ab, int bb, int i, int j) { return Xv[(ab * k + i) * k4 + bb * k + j]; };
    // warm start: rotate A into the previous iteration's eigenbasis Q0 (A
    // changes little between iterations, so few Jacobi sweeps remain)
    double* Q0g = st->Qsyl[v];
    R* Q0 = S;  // shared copy (S is free until the Sylvester solves)
    const bool warm = st->qsyl_valid != 0;
    for (int e = threadIdx.x; e < kk; e += blockDim.x) {
      int i = e / k, j = e % k;
      T2[e] = R(0.5 * (XB(0, 0, i, j) + XB(0, 0, j, i)));
      Q0[e] = warm ? R(Q0g[e]) : R(0);
    }
    __syncthreads();
    if (warm) {
      for (int e = threadIdx.x; e < kk; e += blockDim.x) {  // T = A Q0
        int i = e / k, j = e % k;
        R sum = 0;
        for (int q = 0; q < k; ++q) sum += T2[i * k + q] * Q0[q * k + j];
        T[e] = sum;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < kk; e += blockDim.x) {  // A' = Q0^T T
        int i = e / k, j = e % k;
        R sum = 0;
        for (int q = 0; q < k; ++q) sum += Q0[q * k + i] * T[q * k + j];
        A[e] = sum;
      }
    } else {
      for (int e = threadIdx.x; e < kk; e += blockDim.x) A[e] = T2[e];
    }
    __syncthreads();
    if (threadIdx.x < 32) warp_jacobi<R>(A, T2, lam, k);  // A' = J diag(lam) J^T, J in T2
    __syncthreads();
    if (warm) {
      for (int e = threadIdx.x; e < kk; e += blockDim.x) {  // Q = Q0 J
        int i = e / k, j = e % k;
        R sum = 0;
        for (int q = 0; q < k; ++q) sum += Q0[i * k + q] * T2[q * k + j];
        Q[e] = sum;
      }
    } else {
      for (int e = threadIdx.x; e < kk; e += blockDim.x) Q[e] = T2[e];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kk; e += blockDim.x) Q0g[e] = (double)Q[e];
    __syncthreads();
    // Sylvester solves for the three right-hand sides (C_r + C_r^T,
    // C_r = X[r+1][0]^T) with A = Q diag(lam) Q^T: S_r = Q ((Q^T RHS Q) ./
    // (lam_i + lam_j)) Q^T in R arithmetic.  With R = float one FP64
    // residual correction follows: E = RHS - (A S + S A) in FP64, S += the
    // R-arithmetic solve of A dS + dS A = E.
    double* Sd = Y + 2 * kk;  // 3 kk doubles
    double* A64 = Y;          // sym(X00) in FP64 for the residual (Y is free until the end)
    for (int e = threadIdx.x; e < 3 * kk; e += blockDim.x) {
      int r = e / kk, f = e % kk, i = f / k, j = f % k;
      T2[e] = R(XB(r + 1, 0, i, j) + XB(r + 1, 0, j, i));
      if (r == 0) A64[f] = 0.5 * (XB(0, 0, i, j) + XB(0, 0, j, i));
    }
    __syncthreads();
    for (int pass = 0; pass < (sizeof(R) == 8 ? 1 : 2); ++pass) {
      // T = Q^T RHS ; T2 = (T Q) ./ (lam_i + lam_j) ; T = Q T2 ; S = T Q^T
      for (int e = threadIdx.x; e < 3 * kk; e += blockDim.x) {
        int r = e / kk, f = e % kk, i = f / k, j = f % k;
        R sum = 0;
        for (int q = 0; q < k; ++q) sum += Q[q * k + i] * T2[r * kk + q * k + j];
        T[e] = sum;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < 3 * kk; e += blockDim.x) {
        int r = e / kk, f = e % kk, i = f / k, j = f % k;
        R sum = 0;
        for (int q = 0; q < k; ++q) sum += T[r * kk + i * k + q] * Q[q * k + j];
        T2[e] = sum / (lam[i] + lam[j]);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < 3 * kk; e += blockDim.x) {
        int r = e / kk, f = e % kk, i = f / k, j = f % k;
        R sum = 0;
        for (int q = 0; q < k; ++q) sum += Q[i * k + q] * T2[r * kk + q * k + j];
        T[e] = sum;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < 3 * kk; e += blockDim.x) {
        int r = e / kk, f = e % kk, i = f / k, j = f % k;
        R sum = 0;
        for (int q = 0; q < k; ++q) sum += T[r * kk + i * k + q] * Q[j * k + q];
        Sd[e] = (pass == 0 ? 0.0 : Sd[e]) + (double)sum;
      }
      __syncthreads();
      if (sizeof(R) == 8) break;
      if (pass == 0) {
        // residual in FP64: E = RHS - (A S + S A), A = sym(X00)
        for (int e = threadIdx.x; e < 3 * kk; e += blockDim.x) {
          int r = e / kk, f = e % kk, i = f / k, j = f % k;
          const double* Sr = Sd + r * kk;
          double sum = XB(r + 1, 0, i, j) + XB(r + 1, 0, j, i);
          for (int q = 0; q < k; ++q) sum -= A64[i * k + q] * Sr[q * k + j] + Sr[i * k + q] * A64[q * k + j];
          T2[e] = R(sum);
        }
        __syncthreads();
      }
    }
    for (int e = threadIdx.x; e < 3 * kk; e += blockDim.x) {
      S[e] = R(Sd[e]);
      st->S[v][e / kk][e % kk] = Sd[e];
    }
    __syncthreads();
    const double* Sg = Sd;
    const double* Se = Sd + kk;
    const double* So = Sd + 2 * kk;
    // Y0 = X00 Sg, Y1 = X00 So (FP64)
    for (int e = threadIdx.x; e < 2 * kk; e += blockDim.x) {
      int r = e / kk, f = e % kk, i = f / k, j = f % k;
      const double* Sw = r == 0 ? Sg : So;
      double sum = 0;
      for (int q = 0; q < k; ++q) sum += XB(0, 0, i, q) * Sw[q * k + j];
      Y[e] = sum;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kk; e += blockDim.x) {
      int i = e / k, j = e % k;
      const double dg = (i == j) ? 1.0 : 0.0;
      const double sg = Sg[e], se = Se[e];
      const double sgt = Sg[j * k + i], sot = So[j * k + i];
      // terms: tr X[a][b]; tr(X[a][0] Sw) = sum X[a][0]_ij Sw_ji; tr(Su^T X[0][b]); tr(Su^T Y)
      const double x11 = dg * XB(1, 1, i, i), x13 = dg * XB(1, 3, i, i);
      const double x21 = dg * XB(2, 1, i, i), x23 = dg * XB(2, 3, i, i);
      acc[0] += x11 - XB(1, 0, i, j) * sgt - sg * XB(0, 1, i, j) + sg * Y[e];
      acc[1] += x13 - XB(1, 0, i, j) * sot - sg * XB(0, 3, i, j) + sg * Y[kk + e];
      acc[2] += x21 - XB(2, 0, i, j) * sgt - se * XB(0, 1, i, j) + se * Y[e];
      acc[3] += x23 - XB(2, 0, i, j) * sot - se * XB(0, 3, i, j) + se * Y[kk + e];
      acc[4] += x11 - sg * XB(0, 1, i, j);
      acc[5] += x21 - se * XB(0, 1, i, j);
    }
    __syncthreads();
  }
  blk_sum<6>(acc, red);
  __shared__ int last;
  if (threadIdx.x == 0) {
    for (int q = 0; q < 6; ++q) st->dacc[v][q] = acc[q];
    __threadfence();
    last = atomicAdd(&st->dcount, 1) == a.nviews - 1;
  }
  __syncthreads();
  if (!last) return;
  if (threadIdx.x == 0) {
    __threadfence();
    // every view's sums at once, from L2 (the other CTA's stores are visible
    // there after its fence and our atomic)
    double da[2][6];
#pragma unroll
    for (int w = 0; w < 2; ++w)
#pragma unroll
      for (int q = 0; q < 6; ++q) da[w][q] = w < a.nviews ? __ldcg(&st->dacc[w][q]) : 0.0;
    for (int q = 0; q < 6; ++q) {
      acc[q] = 0;
      for (int w = 0; w < a.nviews; ++w) acc[q] += da[w][q];  // view order: deterministic
    }
    st->dcount = 0;
  }
  const double gg = acc[0], g_Tg = acc[1], Te_g = acc[2], Te_Tg = acc[3], dfg = acc[4], dfTe = acc[5];
  if (threadIdx.x == 0) {
    // the state's scalars in one batch of loads (each would otherwise wait
    // for the stores before it)
    const int first = st->first, it = st->iter;
    const double t_prev = st->t_prev, df_prev = st->df_prev, f_cur = st->f, t_cur = st->t;
    const double gtol = st->gtol, gn0_old = st->gn0;
    double beta = 0;
    if (!first) {
      double num = gg - g_Tg, den = Te_g - Te_Tg;
      beta = den != 0.0 ? fmax(0.0, num / den) : 0.0;
    }
    double df = -dfg + beta * dfTe;
    if (df >= 0) {
      beta = 0;
      df = -gg;
    }
    double gn = sqrt(fmax(gg, 0.0));
    const double gn0 = first ? gn : gn0_old;
    if (first) {
      st->gn0 = gn;
      st->t0 = 1.0 / gn;
    } else {
      st->t0 = t_prev * df_prev / df;
    }
    st->beta = beta;
    st->df = df;
    st->gn = gn;
    if (a.history != nullptr && it <= a.max_iter) {
      a.history[3 * it + 0] = f_cur;
      a.history[3 * it + 1] = gn;
      a.history[3 * it + 2] = first ? 0.0 : t_cur;
    }
    st->first = 0;
    st->force_zero_step = 0;
    st->qsyl_valid = 1;
    if (!(gn > gtol * gn0)) {
      st->done = 1;
      st->status = GBCCA_OK;
    } else if (it >= a.max_iter) {
      st->done = 1;
      st->status = GBCCA_ERR_MAXITER;
    }
  }
}

// ========================================================== new direction
struct NewArgs {
  DevState* st;
  int k, nviews;
  double* Phi[2];
  double* Meta[2];
  double* gold[2];
  double* Mgold[2];
  const double* LL[2];
  const double* RR[2];
  int d[2];
};

__global__ void newdir_kernel(NewArgs a) {
  DevState* st = a.st;
  if (st->done) return;
  const int v = blockIdx.y;
  const int k = a.k, k4 = 4 * k;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;  // (row j, column c)
  const int j = e / k, c = e - j * k;
  if (j >= a.d[v]) return;
  const double* L = a.LL[v] + (int64_t)j * k4;
  const double* R = a.RR[v] + (int64_t)j * k4;
  const double* Sg = st->S[v][0];
  const double* Se = st->S[v][1];
  const double beta = st->beta;
  double wg = 0, bg = 0, we = 0, be = 0;
  for (int q = 0; q < k; ++q) {
    wg += L[q] * Sg[q * k + c];
    bg += R[q] * Sg[q * k + c];
    we += L[q] * Se[q * k + c];
    be += R[q] * Se[q * k + c];
  }
  const double g = L[k + c] - wg;          // grad = xi - Wn Sg
  const double Mg = R[k + c] - bg;         // M grad = egrad - BU Sg
  const double Te = L[2 * k + c] - we;     // T eta = eta - Wn Se
  const double MTe = R[2 * k + c] - be;    // M T eta = M eta - BU Se
  a.gold[v][(int64_t)j * k + c] = g;
  a.Mgold[v][(int64_t)j * k + c] = Mg;
  a.Phi[v][(int64_t)j * 2 * k + k + c] = -g + beta * Te;
  a.Meta[v][(int64_t)j * k + c] = -Mg + beta * MTe;
}

// ===================================================== Rayleigh-Ritz (end)
// From the Grams of [X U, Y V] (or [Xhat W]) at the final point: CCA
// C = Lx^{-1} (U^T Sxy V) Ly^{-T}, SVD via the eigenvectors of C^T C; FDA
// eigen of L^{-1} (W^T S_B W) L^{-T}.  Rotations rot_v map the point to the
// canonical weights; a sign convention makes the largest-magnitude entry of
// each column of U (W) positive.
struct RRArgs {
  DevState* st;
  const double* Gram;     // pass Gram: P_U block at column offx, Q_V block at offy
  int gnc, offx, offy;    // row stride and block offsets of Gram
  const double* phipart;  // [view][nblk][2k x 2k] Gram of Phi (U^T U in the corner)
  int nblk, k, kind, l;
  const double* YPhi;     // FDA (l x 2k)
  int m0;                 // subspace: k (columns U) or 2k (columns [U, eta])
  int check;              // 1: the convergence check of option rtol, at the
                          // start of every `every`-th iteration (a failed
                          // factorization clears rr_ok and leaves the status)
  int every;
};

// Rayleigh-Ritz on span(Phi_v[:, :m]) per view: m = 2k uses the point and
// the last search direction ([U, eta], [V, eta_V]; the pass Grams of the
// final point hold every product needed), a larger subspace than the point
// alone, so its Ritz values are at least as close to the canonical
// correlations; when that Gram is numerically rank deficient (eta ~ 0 or
// nearly dependent on U: a pivot below 1e-12 of the largest diagonal) the
// kernel falls back to m = k.
__global__ void rr_kernel(RRArgs a) {
  extern __shared__ double rsm[];
  DevState* st = a.st;
  // uniform over the CTA: a check runs at iterations every, 2 every, ... only
  if (a.check && (st->done || st->force_zero_step || st->iter == 0 || st->iter % a.every != 0)) return;
  const int k = a.k, k2 = 2 * k, mm0 = a.m0 * a.m0;
  double* Gx = rsm;
  double* Gy = Gx + mm0;
  double* C = Gy + mm0;
  double* Lxi = C + mm0;
  double* Lyi = Lxi + mm0;
  double* T1 = Lyi + mm0;
  double* T2 = T1 + mm0;
  double* Q = T2 + mm0;
  double* lam = Q + mm0;
  double* rot = lam + 2 * kMaxK;
  double* phig = rot + 100;  // 2 x (2k)^2
  __shared__ int s_ok;
  const int nv = a.kind == kCCA ? 2 : 1;
  for (int v = 0; v < nv; ++v) sum_blocks(a.phipart + (int64_t)v * a.nblk * 4 * k * k, a.nblk, 4 * k * k, phig + v * 4 * k * k);
  const int NC = a.gnc, ox = a.offx, oy = a.offy;
  int m = a.m0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const int mm = m * m;
    for (int e = threadIdx.x; e < mm; e += blockDim.x) {
      int i = e / m, j = e % m;
      Gx[e] = a.Gram[(ox + i) * NC + ox + j] + st->lam[0] * phig[i * k2 + j];
      if (a.kind == kCCA) {
        Gy[e] = a.Gram[(oy + i) * NC + oy + j] + st->lam[1] * phig[4 * k * k + i * k2 + j];
        C[e] = a.Gram[(ox + i) * NC + oy + j];
      } else {
        double s = 0;
        for (int c = 0; c < a.l; ++c) s += a.YPhi[c * k2 + i] * a.YPhi[c * k2 + j];
        C[e] = s;
      }
    }
    __syncthreads();
    // largest diagonals, for the rank test after the factorization
    if (threadIdx.x == 0) {
      double dx = 0, dy = 0;
      for (int i = 0; i < m; ++i) {
        dx = fmax(dx, Gx[i * m + i]);
        if (a.kind == kCCA) dy = fmax(dy, Gy[i * m + i]);
      }
      T1[0] = dx;
      T1[1] = dy;
    }
    __syncthreads();
    const double dxmax = T1[0], dymax = T1[1];
    __syncthreads();
    bool ok = blk_chol(Gx, m);
    if (a.kind == kCCA) ok = blk_chol(Gy, m) && ok;
    if (threadIdx.x == 0) {
      bool full = ok;
      for (int i = 0; i < m && full; ++i) {
        if (Gx[i * m + i] * Gx[i * m + i] < 1e-12 * dxmax) full = false;
        if (a.kind == kCCA && Gy[i * m + i] * Gy[i * m + i] < 1e-12 * dymax) full = false;
      }
      s_ok = full ? 1 : (ok ? 2 : 0);  // 1: full rank, 2: factored but near rank deficient
    }
    __syncthreads();
    if (s_ok == 1 || m == k) {
      if (s_ok == 0) {
        if (threadIdx.x == 0) {
          if (!a.check) st->status = GBCCA_ERR_NOT_SPD;
          st->rr_ok = 0;
        }
        return;
      }
      break;
    }
    m = k;  // fall back to the point alone
    __syncthreads();
  }
  blk_lower_inv(Gx, Lxi, m);
  if (a.kind == kCCA) blk_lower_inv(Gy, Lyi, m);
  else
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) Lyi[e] = Lxi[e];
  __syncthreads();
  blk_mm(Lxi, false, C, false, T1, m, m, m, m, m);   // Lx^{-1} C
  blk_mm(T1, false, Lyi, true, C, m, m, m, m, m);    // ... Ly^{-T}  => whitened cross (or FDA matrix)
  if (a.kind == kCCA) {
    blk_mm(C, true, C, false, T1, m, m, m, m, m);    // C^T C
  } else {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      int i = e / m, j = e % m;
      T1[e] = 0.5 * (C[i * m + j] + C[j * m + i]);
    }
    __syncthreads();
  }
  blk_jacobi(T1, Q, lam, m, rot);                    // right singular vectors (CCA) / eigvecs (FDA), descending
  // the leading k: CCA sigma_i = ||C q_i||, left vectors a_i = C q_i / sigma_i
  if (a.kind == kCCA) {
    blk_mm(C, false, Q, false, T2, m, m, k, m, m);   // C Q[:, :k] (columns a_i sigma_i), m x k
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      double s = 0;
      for (int r = 0; r < m; ++r) s += T2[r * k + i] * T2[r * k + i];
      st->sigma[i] = sqrt(s);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * k; e += blockDim.x) {
      int c = e % k;
      double sg = st->sigma[c];
      T2[e] = sg > 0 ? T2[e] / sg : 0.0;
    }
    __syncthreads();
    blk_mm(Lxi, true, T2, false, st->rot[0], m, m, k, m, k);  // rot_x = Lx^{-T} A (m x k)
    blk_mm(Lyi, true, Q, false, st->rot[1], m, m, k, m, m);   // rot_y = Ly^{-T} Q[:, :k]
  } else {
    for (int i = threadIdx.x; i < k; i += blockDim.x) st->sigma[i] = lam[i];
    __syncthreads();
    blk_mm(Lxi, true, Q, false, st->rot[0], m, m, k, m, m);
  }
  if (threadIdx.x == 0) {
    st->rr_m = m;
    st->rr_ok = 1;
  }
}

// Convergence check on the Ritz values (option rtol): row idx of the history
// receives the values the last Rayleigh-Ritz step left in st->sigma; when
// every value changed by less than rtol (relative) since the previous check,
// the iteration ends (st->done) with status OK.
// One-sided (Hestenes) Jacobi SVD of an m x m matrix (m <= 32) by one warp in
// FP32 registers: lane c holds column c of A and of V; the tournament order
// pairs every two columns once per sweep, a pair exchanging its columns by
// shuffles and both lanes computing the same rotation.  On return lane c has
// A[:, c] = sigma_c u_c and V[:, c] = v_c with A_in V = U diag(sigma); for a
// symmetric positive semi-definite input the sigma are its eigenvalues and V
// its eigenvectors.  Column norms are not sorted.  tol: relative size of the
// cosine between two columns below which a pair is left alone.
template <int N>
__device__ void warp_hestenes(float (&a)[N], float (&v)[N], int m, int max_sweeps, float tol) {
  const int lane = threadIdx.x & 31;
  const int mm = m + (m & 1);  // players of the tournament (a bye when m is odd)
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    float worst = 0.f;
    for (int r = 0; r < mm - 1; ++r) {
      // partner of this lane in round r (circle method; player 0 fixed)
      int partner = -1;
      for (int i = 0; i < mm / 2; ++i) {
        const int pa = (i == 0) ? 0 : 1 + ((i - 1 + r) % (mm - 1));
        const int pb = 1 + ((mm - 2 - i + r) % (mm - 1));
        if (pa == lane) partner = pb;
        if (pb == lane) partner = pa;
      }
      const bool active = lane < m && partner >= 0 && partner < m;
      const int src = active ? partner : lane;
      float b[N], vb[N];
#pragma unroll
      for (int q = 0; q < N; ++q) {
        b[q] = __shfl_sync(0xffffffffu, a[q], src);
        vb[q] = __shfl_sync(0xffffffffu, v[q], src);
      }
      if (active) {
        // the pair (p, q) with p < q: both lanes form alpha, beta, gamma in
        // the same order, so they compute the same rotation
        const bool lo = lane < partner;
        float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
        for (int q = 0; q < N; ++q) {
          const float xp = lo ? a[q] : b[q], xq = lo ? b[q] : a[q];
          al = fmaf(xp, xp, al);
          be = fmaf(xq, xq, be);
          ga = fmaf(xp, xq, ga);
        }
        const float den = sqrtf(al * be);
        if (den > 0.f && fabsf(ga) > tol * den) {
          worst = fmaxf(worst, fabsf(ga) / den);
          const float zeta = (be - al) / (2.f * ga);
          const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float c = rsqrtf(1.f + t * t), sn = c * t;
#pragma unroll
          for (int q = 0; q < N; ++q) {
            // column p <- c p - s q; column q <- s p + c q
            a[q] = lo ? c * a[q] - sn * b[q] : sn * b[q] + c * a[q];
            v[q] = lo ? c * v[q] - sn * vb[q] : sn * vb[q] + c * v[q];
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if (worst <= tol) break;
  }
}

// Ritz values for the convergence check (option rtol), by one warp: the
// Rayleigh-Ritz problem of span([U, eta]) x span([V, eta_V]) (CCA; FDA:
// span([W, eta])) from the pass Grams of the current point.  Cholesky of the
// two m x m Grams (pivots by Newton reciprocal square roots), two triangular
// solves for the whitened cross matrix Z = L_x^{-1} C L_y^{-T}, T = Z^T Z (FDA:
// the symmetric Z itself), FP32 Jacobi vectors of T and FP64 Rayleigh
// quotients with them (second-order accurate in the vectors).  Writes
// st->sigma[0 .. k) and st->rr_ok; gated like the check.
inline size_t ritz_values_smem(int k) {
  const size_t m = 2 * (size_t)k;
  return sizeof(double) * (4 * m * m + 2 * m) + sizeof(float) * (2 * m * m + m);
}

struct RitzArgs {
  DevState* st;
  const double* Gram;     // pass Gram, row stride gnc
  int gnc, offx, offy;
  const double* phig;     // [view][2k x 2k] Gram of Phi (summed)
  const double* YPhi;     // FDA (l x 2k)
  int k, kind, l, every;
};

__global__ void __launch_bounds__(32) ritz_values_kernel(RitzArgs a) {
  DevState* st = a.st;
  // runs beside the rest of the iteration: gated on the iteration count
  // taken when the pass finished, not on the live counters
  if (st->check_iter == 0 || st->check_iter % a.every != 0) return;
  constexpr int kM2 = 2 * kMaxK > 32 ? 32 : 2 * kMaxK;  // register columns (m <= 32 here)
  const int lane = threadIdx.x, k = a.k, m = 2 * k, k2 = 2 * k;
  extern __shared__ double rz[];  // ritz_values_smem(k) bytes
  double* Lx = rz;
  double* Ly = Lx + m * m;
  double* Cm = Ly + m * m;
  double* T = Cm + m * m;
  double* ix = T + m * m;
  double* iy = ix + m;
  float* Tf = reinterpret_cast<float*>(iy + m);
  float* Qf = Tf + m * m;
  float* lf = Qf + m * m;
  const bool cca = a.kind == kCCA;
  for (int e = lane; e < m * m; e += 32) {
    const int i = e / m, j = e - i * m;
    Lx[e] = a.Gram[(a.offx + i) * a.gnc + a.offx + j] + st->lam[0] * a.phig[i * k2 + j];
    if (cca) {
      Ly[e] = a.Gram[(a.offy + i) * a.gnc + a.offy + j] + st->lam[1] * a.phig[k2 * k2 + i * k2 + j];
      Cm[e] = a.Gram[(a.offx + i) * a.gnc + a.offy + j];
    } else {
      double sb = 0;
      for (int c = 0; c < a.l; ++c) sb += a.YPhi[c * k2 + i] * a.YPhi[c * k2 + j];
      Cm[e] = sb;
    }
  }
  __syncwarp();
  // Cholesky (lower), right-looking; the reciprocals of the pivots kept
  bool ok = true;
  for (int v = 0; v < (cca ? 2 : 1); ++v) {
    double* A = v == 0 ? Lx : Ly;
    double* inv = v == 0 ? ix : iy;
    for (int j = 0; j < m; ++j) {
      const double dj = A[j * m + j];
      if (!(dj > 0.0)) ok = false;
      const double r = dj > 0.0 ? rsqrt_nr(dj) : 0.0;
      __syncwarp();
      for (int i = j + lane; i < m; i += 32) A[i * m + j] *= r;  // L_jj = d r, L_ij = a_ij r
      if (lane == 0) inv[j] = r;  // 1 / L_jj
      __syncwarp();
      for (int e = lane; e < (m - j - 1) * (m - j - 1); e += 32) {
        const int i = j + 1 + e / (m - j - 1), c = j + 1 + e % (m - j - 1);
        if (c <= i) A[i * m + c] -= A[i * m + j] * A[c * m + j];
      }
      __syncwarp();
    }
  }
  if (!cca) {
    for (int e = lane; e < m * m; e += 32) Ly[e] = Lx[e];
    for (int j = lane; j < m; j += 32) iy[j] = ix[j];
    __syncwarp();
  }
  if (!ok) {
    if (lane == 0) st->rr_ok = 0;
    return;
  }
  // X = L_x^{-1} C (column c of C per lane), into Cm
  for (int c = lane; c < m; c += 32)
    for (int i = 0; i < m; ++i) {
      double s = Cm[i * m + c];
      for (int q = 0; q < i; ++q) s -= Lx[i * m + q] * Cm[q * m + c];
      Cm[i * m + c] = s * ix[i];
    }
  __syncwarp();
  // Z = X L_y^{-T}: row r of X per lane (solve L_y z = x_r^T), into Cm
  for (int r = lane; r < m; r += 32)
    for (int i = 0; i < m; ++i) {
      double s = Cm[r * m + i];
      for (int q = 0; q < i; ++q) s -= Ly[i * m + q] * Cm[r * m + q];
      Cm[r * m + i] = s * iy[i];
    }
  __syncwarp();
  // FDA: the symmetric part of Z (its eigenvalues); CCA: Z (its singular
  // values).  FP32 one-sided Jacobi for the vectors V (lane c: column c), then
  // FP64 Rayleigh quotients ||Z v||^2 / ||v||^2 (CCA) or v^T Z v / v^T v (FDA)
  if (!cca) {
    for (int e = lane; e < m * m; e += 32) {
      const int i = e / m, j = e - i * m;
      T[e] = 0.5 * (Cm[i * m + j] + Cm[j * m + i]);
    }
    __syncwarp();
  }
  const double* Zs = cca ? Cm : T;
  if (m > kM2) {
    // wider than a warp (k > 16): two-sided FP32 Jacobi of Z^T Z (CCA) or
    // of the symmetric part (FDA) in shared memory, FP64 Rayleigh quotients
    for (int e = lane; e < m * m; e += 32) {
      const int i = e / m, j = e - i * m;
      double t = 0;
      if (cca) {
        for (int r = 0; r < m; ++r) t += Cm[r * m + i] * Cm[r * m + j];
        T[e] = t;
      } else {
        t = T[e];
      }
      Tf[e] = (float)t;
    }
    __syncwarp();
    warp_jacobi<float>(Tf, Qf, lf, m, 8, 1e-10f);
    __syncwarp();
    for (int i = lane; i < k; i += 32) {
      double num = 0, den = 0;
      for (int r = 0; r < m; ++r) {
        const double qr = (double)Qf[r * m + i];
        double t = 0;
        for (int c = 0; c < m; ++c) t += T[r * m + c] * (double)Qf[c * m + i];
        num += qr * t;
        den += qr * qr;
      }
      const double rq = den > 0 ? num / den : 0.0;
      st->sigma[i] = cca ? sqrt(fmax(rq, 0.0)) : rq;
    }
    __syncwarp();
    if (lane == 0) st->rr_ok = 1;
    return;
  }
  float av[kM2], vv[kM2];
#pragma unroll
  for (int q = 0; q < kM2; ++q) {
    av[q] = (lane < m && q < m) ? (float)Zs[q * m + lane] : 0.f;
    vv[q] = (q == lane) ? 1.f : 0.f;
  }
  warp_hestenes<kM2>(av, vv, m, 12, 1e-6f);
  // one FP64 Rayleigh quotient per lane (column c of V)
  double rq = -1.0;
  if (lane < m) {
    double num = 0, den = 0;
    for (int r = 0; r < m; ++r) {
      double zr = 0;
#pragma unroll
      for (int q = 0; q < kM2; ++q)
        if (q < m) zr += Zs[r * m + q] * (double)vv[q];
      num += cca ? zr * zr : (double)vv[r] * zr;
    }
#pragma unroll
    for (int q = 0; q < kM2; ++q)
      if (q < m) den += (double)vv[q] * (double)vv[q];
    rq = den > 0 ? num / den : 0.0;
  }
  // the k largest, in descending order: rank of each lane's value
  int rank = 0;
  for (int j = 0; j < m; ++j) {
    const double o = __shfl_sync(0xffffffffu, rq, j);
    if (o > rq || (o == rq && j < lane)) ++rank;
  }
  if (lane < m && rank < k) st->sigma[rank] = cca ? sqrt(fmax(rq, 0.0)) : rq;
  __syncwarp();
  if (lane == 0) st->rr_ok = 1;
}

// Two consecutive small changes are required: a single one can be a pause of
// the iteration rather than convergence.  Runs right after the Rayleigh-Ritz
// step of the check (same gate); when it ends the iteration the remaining
// kernels of the iteration return at once, so the point is the one whose
// values passed the check and the final refinement reproduces them.
__global__ void ritz_check_kernel(DevState* st, double* hist, int len, int k, double rtol, int every) {
  if (threadIdx.x != 0 || st->check_iter == 0 || st->check_iter % every != 0) return;
  const int idx = st->check_iter / every - 1;
  if (!st->rr_ok || idx >= len) return;
  // the change of every value relative to the largest one (the scale of the
  // objective sum mu_i sigma_i and of the accuracy measure max |d sigma| /
  // max sigma): small values, whose relative rounding noise is larger, do
  // not hold the rule back
  double worst = 0, top = 0;
  for (int i = 0; i < k; ++i) top = fmax(top, fabs(st->sigma[i]));
  for (int i = 0; i < k; ++i) {
    const double s = st->sigma[i];
    hist[(int64_t)idx * k + i] = s;
    if (idx > 0) worst = fmax(worst, fabs(s - hist[(int64_t)(idx - 1) * k + i]) / fmax(top, 1e-300));
  }
  st->ritz_checks = idx + 1;
  const bool small = idx > 0 && hist[(int64_t)(idx - 1) * k] != 0.0 && worst < rtol;
  st->ritz_small = small ? st->ritz_small + 1 : 0;
  if (st->ritz_small >= 2) st->ritz_stop = 1;
}

// Before the Ritz branch forks: the iteration count at this pass (0 when
// there is nothing to check: a finished solve or the qf_B step).
__global__ void ritz_snap_kernel(DevState* st) {
  st->check_iter = (st->done || st->force_zero_step) ? 0 : st->iter;
}

// After the Ritz branch joins: a met rule ends the solve.
__global__ void ritz_stop_kernel(DevState* st) {
  if (st->ritz_stop && !st->done) st->done = 1;
}

// out_v (d x k) = Phi_v[:, :m] rot_v (m = the Rayleigh-Ritz subspace used),
// then the sign convention.
__global__ void rr_apply_kernel(DevState* st, const double* Phi, int d, int k, int v, double* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  const int m = st->rr_m;
  for (int c = 0; c < k; ++c) {
    double s = 0;
    for (int q = 0; q < m; ++q) s += Phi[(int64_t)j * 2 * k + q] * st->rot[v][q * k + c];
    out[(int64_t)j * k + c] = s;
  }
}

// sign[c] from view 0: +1 if the largest-magnitude entry of column c is > 0
// Sign convention: the entry of largest magnitude of u_c (first one on ties)
// is made positive, v_c flips with it.  One warp per column.
__global__ void sign_fix_kernel(double* U, int dx, double* V, int dy, int k) {
  const int c = blockIdx.x, lane = threadIdx.x;
  if (c >= k) return;
  double best = 0;
  int bj = 0x7fffffff;
  for (int j = lane; j < dx; j += 32) {
    const double u = U[(int64_t)j * k + c];
    if (fabs(u) > fabs(best)) {
      best = u;
      bj = j;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
    if (fabs(ob) > fabs(best) || (fabs(ob) == fabs(best) && oj < bj)) {
      best = ob;
      bj = oj;
    }
  }
  if (best < 0) {
    for (int j = lane; j < dx; j += 32) U[(int64_t)j * k + c] = -U[(int64_t)j * k + c];
    if (V != nullptr)
      for (int j = lane; j < dy; j += 32) V[(int64_t)j * k + c] = -V[(int64_t)j * k + c];
  }
}

__global__ void copy_sigma_kernel(const DevState* st, double* out, int k) {
  if (threadIdx.x < k) out[threadIdx.x] = st->sigma[threadIdx.x];
}

// FDA: Yhat Phi (l x 2k)
__global__ void yphi_kernel(const DevState* st, const double* Yhat, const double* Phi, int l, int d, int k2,
                            double* YPhi, int check_done) {
  if (check_done && st->done) return;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= l * k2) return;
  int c = e / k2, q = e % k2;
  double s = 0;
  for (int j = 0; j < d; ++j) s += Yhat[(int64_t)c * d + j] * Phi[(int64_t)j * k2 + q];
  YPhi[e] = s;
}

// ============================================================== driver
namespace {

int minv(Plan& p, int v, cudaStream_t st) {
  View& w = p.v[v];
  const int k = p.k, k2 = 2 * k, k4 = 4 * k;
  // tmp = R^{-T} RR[:, 0:2k]; LL[:, 0:2k] = R^{-1} tmp
  if (p.dtype == GBCCA_FP64) {
    GB_TRY(mat_thin<double>(w.Rinv, w.d, w.d, true, true, w.RR, k4, w.tmp, k2, k2, p.mt_part, st));
    GB_TRY(mat_thin<double>(w.Rinv, w.d, w.d, false, true, w.tmp, k2, w.LL, k4, k2, p.mt_part, st));
  } else {
    GB_TRY(mat_thin<float>(w.Rinv32, w.d, w.d, true, true, w.RR, k4, w.tmp, k2, k2, p.mt_part, st));
    GB_TRY(mat_thin<float>(w.Rinv32, w.d, w.d, false, true, w.tmp, k2, w.LL, k4, k2, p.mt_part, st));
  }
  return GBCCA_OK;
}

int phigram(Plan& p, cudaStream_t st, const int* done, double* out = nullptr) {
  const int k2 = 2 * p.k;
  return thin_gram(p, p.v[0].Phi, p.nviews > 1 ? p.v[1].Phi : nullptr, k2, p.v[0].Phi,
                   p.nviews > 1 ? p.v[1].Phi : nullptr, k2, k2, k2, p.phipart, st, done, out);
}

int yphi(Plan& p, cudaStream_t st, int check_done) {
  if (p.kind != kLDA) return GBCCA_OK;
  int len = p.l * 2 * p.k;
  yphi_kernel<<<ceil_div(len, 128), 128, 0, st>>>(p.st, p.Yhat, p.v[0].Phi, p.l, p.D, 2 * p.k, p.YPhi, check_done);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

int thin_blocks(const Plan& p) {
  int dmax = 0;
  for (int v = 0; v < p.nviews; ++v) dmax = std::max(dmax, p.v[v].d);
  return ceil_div(dmax, kThinRows);
}

}  // namespace

// Everything of one iteration after its data pass (the pass outputs G and
// Gram are in place).
int iteration_post(Plan& p, bool low, cudaStream_t st) {
  const int k = p.k, kk = k * k;
  const int* done = &p.st->done;
  if (p.pass_forked) {
    // the Phi Gram (Phi is final once the pass has rounded it) on the side
    // branch, beside the reduction and the Gram of the pass on `st`
    GB_CUDA(cudaStreamWaitEvent(p.side_stream, p.pass_fork, 0));
    GB_TRY(phigram(p, p.side_stream, done, p.phired));
    GB_CUDA(cudaEventRecord(p.pass_join, p.side_stream));
    GB_CUDA(cudaStreamWaitEvent(st, p.pass_join, 0));
    p.pass_forked = false;
  } else {
    GB_TRY(phigram(p, st, done, p.phired));
  }
  GB_TRY(yphi(p, st, 1));
  const bool ritz = p.opt.rtol > 0;
  if (ritz) {
    // convergence check on the Rayleigh-Ritz values of span([U, eta]) at this
    // point (every check_every iterations; the kernels return otherwise), on a
    // branch beside the rest of the iteration: it reads only this pass's
    // Grams, which nothing overwrites before the next pass, and its verdict
    // is applied after the join at the end of the iteration
    ritz_snap_kernel<<<1, 1, 0, st>>>(p.st);
    GB_CHECK_LAUNCH();
    GB_CUDA(cudaEventRecord(p.ritz_fork, st));
    GB_CUDA(cudaStreamWaitEvent(p.side_stream, p.ritz_fork, 0));
    RitzArgs a{};
    a.st = p.st;
    a.Gram = p.Gram;
    a.gnc = p.NC;
    a.offx = 0;
    a.offy = 2 * k;
    a.phig = p.phired;
    a.YPhi = p.YPhi;
    a.k = k;
    a.kind = p.kind;
    a.l = p.l;
    a.every = std::max(1, p.opt.check_every);
    const size_t smem = ritz_values_smem(k);
    GB_CUDA(cudaFuncSetAttribute(ritz_values_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ritz_values_kernel<<<1, 32, smem, p.side_stream>>>(a);
    GB_CHECK_LAUNCH();
    ritz_check_kernel<<<1, 32, 0, p.side_stream>>>(p.st, p.ritz_hist, p.ritz_len, k, p.opt.rtol, a.every);
    GB_CHECK_LAUNCH();
    GB_CUDA(cudaEventRecord(p.ritz_join, p.side_stream));
  }
  {
    LSArgs a{};
    a.st = p.st;
    a.Gram = p.Gram;
    a.phipart = p.phired;
    a.nblk = 1;
    a.NC = p.NC;
    a.k = k;
    a.nviews = p.nviews;
    a.kind = p.kind;
    a.YPhi = p.YPhi;
    a.l = p.l;
    a.history = p.history;
    a.max_iter = p.opt.max_iter;
    a.ls_f = p.ls_f;
    a.ls_L = p.ls_L;
    a.polar = p.opt.retraction == 1 ? 1 : 0;
    size_t smem = sizeof(double) * (9 * kk + 8 * kk + ls_work_doubles(k));
    GB_CUDA(cudaFuncSetAttribute(linesearch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    linesearch_kernel<<<kNTrials, 256, smem, st>>>(a);
    GB_CHECK_LAUNCH();
  }
  {
    UpdArgs a{};
    a.st = p.st;
    a.G = p.G;
    a.NC = p.NC;
    a.k = k;
    a.nviews = p.nviews;
    a.kind = p.kind;
    a.l = p.l;
    a.D = p.D;
    a.Yhat = p.Yhat;
    int dofs = 0, dmax = 0;
    for (int v = 0; v < p.nviews; ++v) {
      a.Phi[v] = p.v[v].Phi;
      a.LL[v] = p.v[v].LL;
      a.RR[v] = p.v[v].RR;
      a.RRh[v] = p.v[v].RRh;
      a.RRl[v] = p.v[v].RRl;
      a.Meta[v] = p.v[v].Meta;
      a.gold[v] = p.v[v].gold;
      a.Mgold[v] = p.v[v].Mgold;
      a.d[v] = p.v[v].d;
      a.dofs[v] = dofs;
      dofs += p.v[v].d;
      dmax = std::max(dmax, p.v[v].d);
    }
    const int rows = std::max(1, 128 / k);
    update_kernel<<<dim3(ceil_div(dmax, rows), p.nviews), rows * k, sizeof(double) * 3 * k * rows, st>>>(a);
    GB_CHECK_LAUNCH();
  }
  if (p.v[0].Minv_hi != nullptr) {
    // LL[:, 0:2k] = M^{-1} RR[:, 0:2k] for every view in one launch
    DfmvArgs m{};
    for (int v = 0; v < p.nviews; ++v)
      m.p[v] = DfmvProblem{p.v[v].Minv_hi, p.v[v].Minv_lo, p.v[v].RRh, p.v[v].RRl, p.v[v].LL,
                           p.v[v].d,       p.v[v].d,       2 * k,       4 * k};
    m.c = 2 * k;
    m.done = done;
    GB_TRY(dfmv(m, p.nviews, st));
  } else {
    for (int v = 0; v < p.nviews; ++v) GB_TRY(minv(p, v, st));
  }
  GB_TRY(thin_gram(p, p.v[0].LL, p.nviews > 1 ? p.v[1].LL : nullptr, 4 * k, p.v[0].RR,
                   p.nviews > 1 ? p.v[1].RR : nullptr, 4 * k, 4 * k, 4 * k, p.crosspart, st, done, p.cross));
  {
    DirArgs a{};
    a.st = p.st;
    a.crosspart = p.cross;
    a.nblk = 1;
    a.k = k;
    a.nviews = p.nviews;
    a.history = p.history;
    a.max_iter = p.opt.max_iter;
    size_t smem = sizeof(double) * (2 * 16 * kk + 5 * kk + 100 + 6 * 256 + 11 * kk + kMaxK);
    if (low) {
      GB_CUDA(cudaFuncSetAttribute(direction_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      direction_kernel<float><<<p.nviews, 256, smem, st>>>(a);
    } else {
      GB_CUDA(cudaFuncSetAttribute(direction_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
      direction_kernel<double><<<p.nviews, 256, smem, st>>>(a);
    }
    GB_CHECK_LAUNCH();
  }
  {
    NewArgs a{};
    a.st = p.st;
    a.k = k;
    a.nviews = p.nviews;
    int dmax = 0;
    for (int v = 0; v < p.nviews; ++v) {
      a.Phi[v] = p.v[v].Phi;
      a.Meta[v] = p.v[v].Meta;
      a.gold[v] = p.v[v].gold;
      a.Mgold[v] = p.v[v].Mgold;
      a.LL[v] = p.v[v].LL;
      a.RR[v] = p.v[v].RR;
      a.d[v] = p.v[v].d;
      dmax = std::max(dmax, p.v[v].d);
    }
    newdir_kernel<<<dim3(ceil_div(dmax * k, 128), p.nviews), 128, 0, st>>>(a);
    GB_CHECK_LAUNCH();
  }
  if (ritz) {
    GB_CUDA(cudaStreamWaitEvent(st, p.ritz_join, 0));
    ritz_stop_kernel<<<1, 1, 0, st>>>(p.st);
    GB_CHECK_LAUNCH();
  }
  return GBCCA_OK;
}

namespace {

// One iteration (or, with force_zero_step set on the device, the qf_B
// normalization of the starting point).
int iteration(Plan& p, bool low, cudaStream_t st, cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr) {
  p.kev0 = e0;
  p.kev1 = e1;
  p.pass_forked = false;
  p.fork_after_pass = true;
  const int prc = fused_pass(p, low, false, st, 0, &p.st->done);
  p.fork_after_pass = false;
  p.kev0 = p.kev1 = nullptr;
  GB_TRY(prc);
  return iteration_post(p, low, st);
}

// A batch of nb iterations launched one by one (pass b of the batch timed
// with event pair b when timing is on).
int run_batch_direct(Plan& p, bool low, int nb, bool timed, cudaStream_t st) {
  for (int b = 0; b < nb; ++b)
    GB_TRY(iteration(p, low, st, timed ? p.ev[2 * b] : nullptr, timed ? p.ev[2 * b + 1] : nullptr));
  return GBCCA_OK;
}

// The same batch replayed from a CUDA graph.  The graph is captured on the
// plan's own stream and holds plan-owned pointers, the data pointers (X, Y,
// labels; the TMA descriptors are captured by value) and the batch shape; it
// is captured again when any of those differ.  Every kernel reads its
// per-iteration state (step, direction, convergence flag) from device memory,
// so one capture serves every batch of every solve.  With pass timing the
// events around the data kernels are captured as external event-record nodes,
// recorded again at every replay.
int run_batch_graph(Plan& p, bool low, int nb, bool timed, cudaStream_t st) {
  const void* key[3] = {p.v[0].Z, p.nviews > 1 ? (const void*)p.v[1].Z : nullptr, (const void*)p.labels};
  const bool same = p.batch_exec != nullptr && p.batch_key_n == nb && p.batch_key_timed == timed &&
                    key[0] == p.batch_key_ptr[0] && key[1] == p.batch_key_ptr[1] && key[2] == p.batch_key_ptr[2];
  if (!same) {
    if (p.batch_exec != nullptr) {
      GB_CUDA(cudaGraphExecDestroy(p.batch_exec));
      p.batch_exec = nullptr;
    }
    if (p.cap_stream == nullptr) GB_CUDA(cudaStreamCreateWithFlags(&p.cap_stream, cudaStreamNonBlocking));
    const long long l0 = g_launches.load();
    GB_CUDA(cudaStreamBeginCapture(p.cap_stream, cudaStreamCaptureModeRelaxed));
    const int rc = run_batch_direct(p, low, nb, timed, p.cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(p.cap_stream, &g);
    if (rc != GBCCA_OK || ec != cudaSuccess) {
      if (g != nullptr) cudaGraphDestroy(g);
      g_launches.fetch_sub(g_launches.load() - l0);
      cudaGetLastError();  // leave no capture error behind for later calls
      if (rc != GBCCA_OK) return rc;
      set_last_error(std::string("capture of the iteration batch: ") + cudaGetErrorString(ec));
      return GBCCA_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&p.batch_exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      p.batch_exec = nullptr;
      cudaGetLastError();
      set_last_error(std::string("instantiation of the iteration batch: ") + cudaGetErrorString(ei));
      return GBCCA_ERR_CUDA;
    }
    // the launches made while capturing ran nothing: count them per replay
    p.batch_launches = g_launches.load() - l0;
    g_launches.fetch_sub(p.batch_launches);
    p.batch_key_n = nb;
    p.batch_key_timed = timed;
    for (int i = 0; i < 3; ++i) p.batch_key_ptr[i] = key[i];
  }
  GB_CUDA(cudaGraphLaunch(p.batch_exec, st));
  g_launches.fetch_add(p.batch_launches);
  return GBCCA_OK;
}

}  // namespace

__global__ void state_init_kernel(DevState* st, double gtol, int max_iter, double lam0, double lam1) {
  st->iter = 0;
  st->done = 0;
  st->status = GBCCA_OK;
  st->stalled = 0;
  st->passes = 0;
  st->ls_trials = 0;
  st->first = 1;
  st->force_zero_step = 1;
  st->t = st->f = st->df = st->t_prev = st->df_prev = st->gn = st->gn0 = st->beta = st->t0 = 0;
  st->gtol = gtol;
  st->max_iter = max_iter;
  st->qsyl_valid = 0;
  st->rr_ok = 0;
  st->ritz_checks = 0;
  st->ritz_small = 0;
  st->check_iter = 0;
  st->ritz_stop = 0;
  st->dcount = 0;
  st->ls_count = 0;
  st->lam[0] = lam0;
  st->lam[1] = lam1;
}

// Starting point in Phi[:, :k] (eta = 0 and all carried vectors zero).
__global__ void start_kernel(const double* src, double* Phi, double* Meta, double* gold, double* Mgold, int d, int k) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  for (int c = 0; c < k; ++c) {
    Phi[(int64_t)j * 2 * k + c] = src[(int64_t)j * k + c];
    Phi[(int64_t)j * 2 * k + k + c] = 0.0;
    Meta[(int64_t)j * k + c] = 0.0;
    gold[(int64_t)j * k + c] = 0.0;
    Mgold[(int64_t)j * k + c] = 0.0;
  }
}

// A kernel that gave up a bounded wait (or found a non-SPD factor) sets the
// plan's error flag; the host reads it with the state after every batch.
int check_flag(Plan& p, gbcca_info* info, cudaStream_t st) {
  if (*p.flag_host == 0) return GBCCA_OK;
  const int f = *p.flag_host;
  *p.flag_host = 0;
  GB_CUDA(cudaMemsetAsync(p.flag, 0, sizeof(int), st));
  GB_CUDA(cudaStreamSynchronize(st));
  const int rc = flag_status(f);
  if (info != nullptr) {
    *info = gbcca_info{};
    info->status = rc;
  }
  return rc;
}

// Device state, weights N and starting point of a solve (the first
// iteration, run by the caller, is the qf_B normalization of the start).
int rcg_begin(Plan& p, const double* mu, double tol, const double* start0, const double* start1, cudaStream_t st) {
  const int k = p.k;
  const double gtol = tol > 0 ? tol : p.opt.gtol;
  state_init_kernel<<<1, 1, 0, st>>>(p.st, gtol, p.opt.max_iter, p.v[0].lam, p.nviews > 1 ? p.v[1].lam : 0.0);
  GB_CHECK_LAUNCH();
  double muh[kMaxK];
  // default weights N = diag(1 + (k - 1 - i) / 100): the solution does not
  // depend on N (Thm 4.1) but the conditioning does (Thm 4.4); near-equal
  // weights make the iteration converge the subspace at the rate of the gap
  // sigma_k - sigma_{k+1}, and the final Rayleigh-Ritz step separates the
  // pairs inside it
  for (int i = 0; i < k; ++i) muh[i] = mu ? mu[i] : 1.0 + 0.01 * (double)(k - 1 - i);
  GB_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(p.st) + offsetof(DevState, mu), muh, sizeof(double) * k,
                          cudaMemcpyHostToDevice, st));
  for (int v = 0; v < p.nviews; ++v) {
    const double* src = p.opt.warm_start ? p.v[v].warm : (v == 0 ? start0 : start1);
    start_kernel<<<ceil_div(p.v[v].d, 128), 128, 0, st>>>(src, p.v[v].Phi, p.v[v].Meta, p.v[v].gold, p.v[v].Mgold,
                                                          p.v[v].d, k);
    GB_CHECK_LAUNCH();
  }
  GB_CUDA(cudaMemsetAsync(p.history, 0, sizeof(double) * 3 * (p.opt.max_iter + 1), st));
  GB_CUDA(cudaMemsetAsync(p.ritz_hist, 0, sizeof(double) * p.ritz_len * k, st));
  return GBCCA_OK;
}

// Rayleigh-Ritz at the final point, outputs, and the report.  FP64 data: over
// span([U, eta]) with the Grams of the plan's FP64 pass (exact products).
// BF16/FP32 data, refine = 1: over span(U) with the Grams of [X U, Y V] from
// an FP64 pass (exact products of the stored data); refine = 2: over
// span([U, eta]) with the Grams of the plan's own pass (FP32 accumulation).
int rcg_finish(Plan& p, double* out0, double* out1, double* vals, gbcca_info* info, double pass_ms, int pass_count,
               cudaStream_t st) {
  const int k = p.k;
  const bool low = p.dtype != GBCCA_FP64;
  const bool exact_refine = low && p.opt.refine != 2;
  if (exact_refine) {
    GB_TRY(fused_pass(p, false, true, st, k, nullptr));
  } else {
    GB_TRY(fused_pass(p, low, false, st, 0, nullptr));
  }
  GB_TRY(phigram(p, st, nullptr));
  GB_TRY(yphi(p, st, 0));
  {
    RRArgs a{};
    a.st = p.st;
    a.Gram = p.Gram;
    if (exact_refine) {
      a.gnc = p.nviews * k;
      a.offx = 0;
      a.offy = k;
    } else {
      a.gnc = p.NC;
      a.offx = 0;
      a.offy = 2 * k;
    }
    a.phipart = p.phipart;
    a.nblk = thin_blocks(p);
    a.k = k;
    a.kind = p.kind;
    a.l = p.l;
    a.YPhi = p.YPhi;
    // the pass Grams of [U, eta] (low-precision pass) allow the 2k subspace;
    // the exact refinement pass forms the U columns only
    a.m0 = exact_refine ? k : 2 * k;
    size_t smem = sizeof(double) * (8 * a.m0 * a.m0 + 2 * kMaxK + 100 + 8 * k * k);
    GB_CUDA(cudaFuncSetAttribute(rr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    rr_kernel<<<1, 256, smem, st>>>(a);
    GB_CHECK_LAUNCH();
  }
  for (int v = 0; v < p.nviews; ++v) {
    double* out = v == 0 ? out0 : out1;
    rr_apply_kernel<<<ceil_div(p.v[v].d, 128), 128, 0, st>>>(p.st, p.v[v].Phi, p.v[v].d, k, v, out);
    GB_CHECK_LAUNCH();
  }
  sign_fix_kernel<<<k, 32, 0, st>>>(out0, p.v[0].d, p.nviews > 1 ? out1 : nullptr, p.nviews > 1 ? p.v[1].d : 0, k);
  GB_CHECK_LAUNCH();
  copy_sigma_kernel<<<1, 32, 0, st>>>(p.st, vals, k);
  GB_CHECK_LAUNCH();
  GB_CUDA(cudaMemcpyAsync(p.st_host, p.st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  GB_CUDA(cudaMemcpyAsync(p.flag_host, p.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  GB_CUDA(cudaStreamSynchronize(st));
  GB_TRY(check_flag(p, info, st));
  const int status = p.st_host->status;
  if (info != nullptr) {
    info->iters = p.st_host->iter;
    info->passes = p.st_host->iter + 2;  // the qf_B pass, one per iteration, the final one
    info->status = status;
    info->stalled = p.st_host->stalled;
    info->grad_norm = p.st_host->gn;
    info->grad_norm0 = p.st_host->gn0;
    info->objective = p.st_host->f;
    info->pass_ms = pass_count > 0 ? pass_ms / pass_count : 0.0;
    info->pass_count = pass_count;
  }
  return status;
}

// Enqueue the state and flag reads of a plan (host mirrors) on `st`.
int read_state_async(Plan& p, cudaStream_t st) {
  GB_CUDA(cudaMemcpyAsync(p.st_host, p.st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  GB_CUDA(cudaMemcpyAsync(p.flag_host, p.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  return GBCCA_OK;
}

int rcg_run(Plan& p, const double* mu, double tol, double* out0, double* out1, double* vals, gbcca_info* info,
            cudaStream_t st) {
  const bool low = p.dtype != GBCCA_FP64;
  GB_TRY(rcg_begin(p, mu, tol, out0, out1, st));
  // qf_B of the start (zero step), then iterations in batches.  With pass
  // timing, event pair b brackets the pass of global iteration index
  // first_index + b (index 0 = the qf_B pass); only passes whose iteration
  // really ran (index <= iterations done) are counted.
  const bool timed = p.nev > 0;
  double pass_ms = 0;
  int pass_count = 0;
  auto harvest = [&](int first_index, int nb, int iters_done) -> int {
    for (int b = 0; b < nb; ++b) {
      if (first_index + b > iters_done) break;
      float ms = 0;
      GB_CUDA(cudaEventElapsedTime(&ms, p.ev[2 * b], p.ev[2 * b + 1]));
      pass_ms += ms;
      ++pass_count;
    }
    return GBCCA_OK;
  };
  GB_TRY(iteration(p, low, st, timed ? p.ev[0] : nullptr, timed ? p.ev[1] : nullptr));
  int launched = 0;
  int batch = std::max(1, p.opt.check_every);
  if (timed) batch = std::min(batch, kMaxTimedBatch);
  int pending_first = 0, pending_n = timed ? 1 : 0;
  while (true) {
    GB_TRY(read_state_async(p, st));
    GB_CUDA(cudaStreamSynchronize(st));
    GB_TRY(check_flag(p, info, st));
    if (timed) GB_TRY(harvest(pending_first, pending_n, p.st_host->iter));
    if (p.st_host->done || launched >= p.opt.max_iter) break;
    pending_first = launched + 1;
    const int nb = std::min(batch, p.opt.max_iter - launched);
    // full batches replay a captured graph; a shorter last batch is launched
    // kernel by kernel (same kernels, same order)
    if (p.opt.graphs && nb == batch)
      GB_TRY(run_batch_graph(p, low, nb, timed, st));
    else
      GB_TRY(run_batch_direct(p, low, nb, timed, st));
    launched += nb;
    pending_n = timed ? nb : 0;
  }
  return rcg_finish(p, out0, out1, vals, info, pass_ms, pass_count, st);
}

// ============================================================ warm start
// CCA: top-k singular pairs of C = R_x^{-T} (X_S^T Y_S) R_y^{-1} by block
// power iteration with CholeskyQR re-orthonormalization (2k columns), then a
// Rayleigh-Ritz step; U~ = R_x^{-1} A_k, V~ = R_y^{-1} B_k (exact CCA of the
// sketched pair, Alg. 1 step 4).  FDA: eigen of G G^T with G = Yhat R^{-1}
// (l x l), W~ = R^{-1} G^T Q_k diag(lambda)^{-1/2} (Alg. 2 step 5).

__global__ void rand_block_kernel(double* B, int d, int c, uint64_t seed) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d * c) return;
  uint64_t r = sm64(seed ^ 0xA5A5A5A5DEADBEEFull, (uint64_t)e);
  B[e] = (double)(r >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

// small Gram (c x c) of a d x c block: reduce partials, Cholesky (ridge for
// safety) -> upper R in out (R^T R = G), and its inverse in out + c*c.
__global__ void small_chol_kernel(const double* part, int nblk, int c, double* out, int* flag) {
  extern __shared__ double ssm[];
  double* G = ssm;
  double* Li = G + c * c;
  sum_blocks(part, nblk, c * c, G);
  double tr = 0;
  for (int i = 0; i < c; ++i) tr += G[i * c + i];
  __syncthreads();
  if (threadIdx.x < c) G[threadIdx.x * c + threadIdx.x] += 1e-14 * tr / c;
  __syncthreads();
  if (c <= 32) {
    // c <= 32: one warp factors G, pivots used through their reciprocals
    if (threadIdx.x < 32) {
      double* invd = Li + c * c;
      const bool ok = warp_chol(G, c, invd);
      if (!ok && threadIdx.x == 0) atomicExch(flag, kFlagNotSpd);
      warp_lower_inv(G, invd, Li, c);
    }
    __syncthreads();
  } else {
    if (!blk_chol(G, c)) {
      if (threadIdx.x == 0) atomicExch(flag, kFlagNotSpd);
    }
    blk_lower_inv(G, Li, c);
  }
  // R^{-1} = (L^{-1})^T
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    int i = e / c, j = e % c;
    out[e] = Li[j * c + i];
  }
}

// B (d x c) <- B Rinv (c x c upper): a CTA stages kApplyRows rows of B in
// shared memory and each thread forms one entry (at most c multiply-adds),
// so the FP64 work spreads over many SMs instead of one chain per row.
constexpr int kApplyRows = 8;
__global__ void __launch_bounds__(kApplyRows * 2 * kMaxK) apply_small_kernel(double* B, int d, int c,
                                                                            const double* Rinv) {
  __shared__ double rows[kApplyRows * 2 * kMaxK];
  const int j0 = blockIdx.x * kApplyRows;
  const int nr = min(kApplyRows, d - j0);
  for (int e = threadIdx.x; e < nr * c; e += blockDim.x) rows[e] = B[(int64_t)j0 * c + e];
  __syncthreads();
  const int e = threadIdx.x;
  if (e >= nr * c) return;
  const int r = e / c, q = e - r * c;
  double s = 0;
  for (int t = 0; t <= q; ++t) s += rows[r * c + t] * Rinv[t * c + q];
  B[(int64_t)(j0 + r) * c + q] = s;
}

// Rayleigh-Ritz of the power iteration: Bsmall = U^T (C V) (c x c), take the
// top-k singular pairs: U A_k, V B_k in out (d x k each).
__global__ void small_svd_kernel(const double* part, int nblk, int c, int k, double* rotU, double* rotV) {
  extern __shared__ double wsm[];
  double* Bm = wsm;
  double* T = Bm + c * c;
  double* Q = T + c * c;
  double* lam = Q + c * c;
  double* rot = lam + 2 * kMaxK;
  sum_blocks(part, nblk, c * c, Bm);
  blk_mm(Bm, true, Bm, false, T, c, c, c, c, c);  // B^T B
  blk_jacobi(T, Q, lam, c, rot);                 // right singular vectors
  blk_mm(Bm, false, Q, false, T, c, c, c, c, c);  // B Q = A Sigma
  for (int e = threadIdx.x; e < c * k; e += blockDim.x) {
    int r = e / k, i = e % k;
    double s = 0;
    for (int q = 0; q < c; ++q) s += T[q * c + i] * T[q * c + i];
    s = sqrt(s);
    rotU[r * k + i] = s > 0 ? T[r * c + i] / s : 0.0;
    rotV[r * k + i] = Q[r * c + i];
  }
}

__global__ void thin_apply_kernel(const double* B, int d, int c, const double* rot, int k, double* out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  for (int i = 0; i < k; ++i) {
    double s = 0;
    for (int q = 0; q < c; ++q) s += B[(int64_t)j * c + q] * rot[q * k + i];
    out[(int64_t)j * k + i] = s;
  }
}

// FDA warm start pieces
__global__ void transpose_kernel(const double* A, int r, int c, double* At) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * c) return;
  int i = e / c, j = e % c;
  At[(int64_t)j * r + i] = A[e];
}

__global__ void fda_warm_kernel(const double* part, int nblk, int l, int k, double* rot) {
  extern __shared__ double fsm[];
  double* K = fsm;
  double* Q = K + l * l;
  double* lam = Q + l * l;
  double* r = lam + kMaxClasses;
  sum_blocks(part, nblk, l * l, K);
  blk_jacobi(K, Q, lam, l, r);
  for (int e = threadIdx.x; e < l * k; e += blockDim.x) {
    int q = e / k, i = e % k;
    rot[e] = lam[i] > 0 ? Q[q * l + i] / sqrt(lam[i]) : 0.0;
  }
}

namespace {

int orth(Plan& p, double* B, int d, int c, double* part, double* small, cudaStream_t st) {
  // Gram of B (d x c) via a one-view thin Gram
  ThinArgs a{};
  a.A[0] = B;
  a.B[0] = B;
  a.lda[0] = c;
  a.ldb[0] = c;
  a.d[0] = d;
  a.ca = c;
  a.cb = c;
  a.nblk = ceil_div(d, kThinRows);
  a.part = part;
  a.done = nullptr;
  size_t smem = sizeof(double) * kThinRows * 2 * c;
  GB_CUDA(cudaFuncSetAttribute(thin_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  thin_gram_kernel<<<dim3(a.nblk, 1), 256, smem, st>>>(a);
  GB_CHECK_LAUNCH();
  small_chol_kernel<<<1, 256, sizeof(double) * (2 * c * c + c), st>>>(part, a.nblk, c, small, p.flag);
  GB_CHECK_LAUNCH();
  apply_small_kernel<<<ceil_div(d, kApplyRows), kApplyRows * 2 * kMaxK, 0, st>>>(B, d, c, small);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

}  // namespace

int warm_start(Plan& p, cudaStream_t st) {
  const int k = p.k;
  if (p.kind == kCCA) {
    View& x = p.v[0];
    View& y = p.v[1];
    const int dx = x.d, dy = y.d;
    const int c = std::min(2 * k, std::min(dx, dy));
    // Cxy = X_S^T Y_S (dx x dy), kept in ws after the Gram partials
    double* Cxy = p.ws + (p.ws_len - (int64_t)dx * dy);
    if (x.SZh != nullptr)
      GB_TRY(gram_df_split(x.SZh, x.SZl, dx, y.SZh, y.SZl, dy, p.s, dx, dy, Cxy, 0.0, p.ws,
                           p.ws_len - (int64_t)dx * dy, st));
    else
      GB_TRY(gram_tn(x.SZ, dx, y.SZ, dy, p.s, dx, dy, Cxy, 0.0, p.ws, p.ws_len - (int64_t)dx * dy, st));
    double* Vb = y.wsU;  // dy x c
    double* Ub = x.wsU;  // dx x c
    double* part = p.crosspart;
    double* small = p.phigram;
    // Products of the power iteration.  FP64 plans: FP64 triangular / dense
    // products.  FP32/BF16 plans: the same products with double-float copies
    // of R_x^{-1}, R_y^{-1}, Cxy and their transposes (~2^-44 relative, at
    // FP32 instruction rates); FP32 copies of R^{-1} (kappa ~ 1e4) give a
    // visibly worse start point and more solver iterations.
    const bool low = p.dtype != GBCCA_FP64 && (c & 1) == 0;
    float* F = reinterpret_cast<float*>(p.ws);
    const int64_t nx = (int64_t)dx * dx, ny = (int64_t)dy * dy, nc = (int64_t)dx * dy;
    float* Rx[2] = {F, F + nx};              // R_x^{-1} hi, lo
    float* RxT[2] = {F + 2 * nx, F + 3 * nx};
    float* Ry[2] = {F + 4 * nx, F + 4 * nx + ny};
    float* RyT[2] = {F + 4 * nx + 2 * ny, F + 4 * nx + 3 * ny};
    float* Cf[2] = {F + 4 * nx + 4 * ny, F + 4 * nx + 4 * ny + nc};
    float* CfT[2] = {F + 4 * nx + 4 * ny + 2 * nc, F + 4 * nx + 4 * ny + 3 * nc};
    if (low) {
      GB_TRY(split_df(x.Rinv, dx, dx, false, Rx[0], Rx[1], st));
      GB_TRY(split_df(x.Rinv, dx, dx, true, RxT[0], RxT[1], st));
      GB_TRY(split_df(y.Rinv, dy, dy, false, Ry[0], Ry[1], st));
      GB_TRY(split_df(y.Rinv, dy, dy, true, RyT[0], RyT[1], st));
      GB_TRY(split_df(Cxy, dx, dy, false, Cf[0], Cf[1], st));
      GB_TRY(split_df(Cxy, dx, dy, true, CfT[0], CfT[1], st));
    }
    auto dmv = [&](float* const* A, int m, int K, const double* B, double* C) {
      float* bh = p.dfx;
      float* bl = p.dfx + (int64_t)K * c;
      GB_TRY(split_rows(B, K, c, c, bh, bl, st));
      DfmvArgs g{};
      g.p[0] = DfmvProblem{A[0], A[1], bh, bl, C, m, K, c, c};
      g.c = c;
      return dfmv(g, 1, st);
    };
    auto rx = [&](bool tr, const double* B, double* C, int cc) {
      if (low && cc == c) return dmv(tr ? RxT : Rx, dx, dx, B, C);
      return mat_thin<double>(x.Rinv, dx, dx, tr, true, B, cc, C, cc, cc, p.mt_part, st);
    };
    auto ry = [&](bool tr, const double* B, double* C, int cc) {
      if (low && cc == c) return dmv(tr ? RyT : Ry, dy, dy, B, C);
      return mat_thin<double>(y.Rinv, dy, dy, tr, true, B, cc, C, cc, cc, p.mt_part, st);
    };
    auto cxy = [&](bool tr, const double* B, double* C) {
      if (low) return tr ? dmv(CfT, dy, dx, B, C) : dmv(Cf, dx, dy, B, C);
      return mat_thin<double>(Cxy, dx, dy, tr, false, B, c, C, c, c, p.mt_part, st);
    };
    rand_block_kernel<<<ceil_div(dy * c, 256), 256, 0, st>>>(Vb, dy, c, p.opt.seed);
    GB_CHECK_LAUNCH();
    GB_TRY(orth(p, Vb, dy, c, part, small, st));
    const int iters = p.opt.warm_iters > 0 ? p.opt.warm_iters : 12;
    for (int it = 0; it <= iters; ++it) {
      // U = orth(R_x^{-T} Cxy R_y^{-1} V)
      GB_TRY(ry(false, Vb, y.wsT, c));
      GB_TRY(cxy(false, y.wsT, x.wsT));
      GB_TRY(rx(true, x.wsT, Ub, c));
      if (it == iters) break;  // Ub = C V (unnormalized) for the Rayleigh-Ritz step
      // V = orth(C^T U) with C = R_x^{-T} Cxy R_y^{-1}: U = C V needs no
      // orthonormalization of its own (span(C^T C V) is the same either way,
      // and one step changes the conditioning of the block only by the
      // spread of the top 2k singular values)
      GB_TRY(rx(false, Ub, x.wsT, c));
      GB_TRY(cxy(true, x.wsT, y.wsT));
      GB_TRY(ry(true, y.wsT, Vb, c));
      GB_TRY(orth(p, Vb, dy, c, part, small, st));
    }
    // Ub = C V: take U0 = orth(Ub) and Bm = U0^T (C V)
    GB_CUDA(cudaMemcpyAsync(x.wsT, Ub, sizeof(double) * dx * c, cudaMemcpyDeviceToDevice, st));
    GB_TRY(orth(p, Ub, dx, c, part, small, st));
    {
      ThinArgs a{};
      a.A[0] = Ub;
      a.B[0] = x.wsT;
      a.lda[0] = c;
      a.ldb[0] = c;
      a.d[0] = dx;
      a.ca = c;
      a.cb = c;
      a.nblk = ceil_div(dx, kThinRows);
      a.part = part;
      size_t smem = sizeof(double) * kThinRows * 2 * c;
      GB_CUDA(cudaFuncSetAttribute(thin_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      thin_gram_kernel<<<dim3(a.nblk, 1), 256, smem, st>>>(a);
      GB_CHECK_LAUNCH();
      double* rotU = small;
      double* rotV = small + c * k;
      size_t sm2 = sizeof(double) * (3 * c * c + 2 * kMaxK + 100);
      GB_CUDA(cudaFuncSetAttribute(small_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
      small_svd_kernel<<<1, 256, sm2, st>>>(part, a.nblk, c, k, rotU, rotV);
      GB_CHECK_LAUNCH();
      // whitened top-k vectors, then back through R^{-1}
      thin_apply_kernel<<<ceil_div(dx, 128), 128, 0, st>>>(Ub, dx, c, rotU, k, x.wsT);
      GB_CHECK_LAUNCH();
      thin_apply_kernel<<<ceil_div(dy, 128), 128, 0, st>>>(Vb, dy, c, rotV, k, y.wsT);
      GB_CHECK_LAUNCH();
      GB_TRY(rx(false, x.wsT, x.warm, k));
      GB_TRY(ry(false, y.wsT, y.warm, k));
    }
    return GBCCA_OK;
  }
  // FDA
  View& x = p.v[0];
  const int d = x.d, l = p.l;
  double* YhT = x.wsT;              // d x l  (wsT has d x 2k >= ... use ws instead when l > 2k)
  double* Gt = p.ws;                // d x l: R^{-T} Yhat^T
  double* YT = p.ws + (int64_t)d * l;
  (void)YhT;
  transpose_kernel<<<ceil_div(l * d, 256), 256, 0, st>>>(p.Yhat, l, d, YT);
  GB_CHECK_LAUNCH();
  GB_TRY(mat_thin<double>(x.Rinv, d, d, true, true, YT, l, Gt, l, l, p.mt_part, st));
  {
    ThinArgs a{};
    a.A[0] = Gt;
    a.B[0] = Gt;
    a.lda[0] = l;
    a.ldb[0] = l;
    a.d[0] = d;
    a.ca = l;
    a.cb = l;
    a.nblk = ceil_div(d, kThinRows);
    a.part = p.crosspart;
    size_t smem = sizeof(double) * kThinRows * 2 * l;
    GB_CUDA(cudaFuncSetAttribute(thin_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    thin_gram_kernel<<<dim3(a.nblk, 1), 256, smem, st>>>(a);
    GB_CHECK_LAUNCH();
    double* rot = p.phigram;  // l x k
    size_t sm2 = sizeof(double) * (2 * l * l + kMaxClasses + 100);
    GB_CUDA(cudaFuncSetAttribute(fda_warm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
    fda_warm_kernel<<<1, 256, sm2, st>>>(p.crosspart, a.nblk, l, k, rot);
    GB_CHECK_LAUNCH();
    double* Wwh = p.ws + 2 * (int64_t)d * l;  // d x k
    thin_apply_kernel<<<ceil_div(d, 128), 128, 0, st>>>(Gt, d, l, rot, k, Wwh);
    GB_CHECK_LAUNCH();
    GB_TRY(mat_thin<double>(x.Rinv, d, d, false, true, Wwh, k, x.warm, k, k, p.mt_part, st));
  }
  return GBCCA_OK;
}

}  // namespace gbcca
