// Small dense FP64 linear algebra for the preconditioner (Sec. 3): the Gram of
// the sketch, its Cholesky factor R (R^T R = (S Z)^T (S Z) + lambda I, the R
// of the QR of [S Z; sqrt(lambda) I]), R^{-1}, and products of d x d factors
// with d x c blocks (the M^{-1} = R^{-1} R^{-T} applications of Table 1).
//
// GB300 executes FP64 at ~1/60 of its FP32 rate, so these kernels spread the
// O(s d^2) and O(d^3) work over many CTAs (split-K Gram, blocked right-looking
// Cholesky, one warp per column of R^{-1}).
#include <mutex>
#include <string>

#include "plan.h"

namespace gbcca {

// ------------------------------------------------------------------- Gram
// C (d1 x d2) = A^T B (+ diag_add on the diagonal), A: m x d1, B: m x d2,
// row-major, FP64.  64 x 64 output tiles, split over K into `ks` partials that
// a second kernel adds in fixed order.
constexpr int kGT = 64, kGK = 16;

__global__ void __launch_bounds__(256)
gram_tn_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ B, int64_t ldb,
               int64_t m, int d1, int d2, int64_t kchunk, double* __restrict__ part) {
  __shared__ double As[kGK][kGT];
  __shared__ double Bs[kGK][kGT];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * kGT, j0 = blockIdx.x * kGT;
  const int64_t k0 = blockIdx.z * kchunk, k1 = min(m, k0 + kchunk);
  double acc[4][4] = {};
  for (int64_t kk = k0; kk < k1; kk += kGK) {
    for (int e = tid; e < kGK * kGT; e += 256) {
      int r = e / kGT, c = e % kGT;
      int64_t row = kk + r;
      As[r][c] = (row < k1 && i0 + c < d1) ? A[row * lda + i0 + c] : 0.0;
      Bs[r][c] = (row < k1 && j0 + c < d2) ? B[row * ldb + j0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kGK; ++r) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[r][ty + 16 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u) b[u] = Bs[r][tx + 16 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] += a[u] * b[w];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      int i = i0 + ty + 16 * u, j = j0 + tx + 16 * w;
      if (i < d1 && j < d2) part[((int64_t)blockIdx.z * d1 + i) * d2 + j] = acc[u][w];
    }
}

// C (d x d) from the split-K partials of a symmetric Gram whose tiles were
// formed on and below the diagonal only: the upper tiles mirror the lower.
__global__ void sum_parts_sym_kernel(const double* __restrict__ part, int nparts, int d, double diag_add,
                                     double* __restrict__ C) {
  const int64_t len = (int64_t)d * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / d), j = (int)(e % d);
    const int64_t src = (i / kGT >= j / kGT) ? e : (int64_t)j * d + i;
    double s = 0;
    for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * len + src];
    if (i == j) s += diag_add;
    C[e] = s;
  }
}

__global__ void sum_parts_kernel(const double* __restrict__ part, int nparts, int64_t len, int d1, int d2,
                                 double diag_add, double* __restrict__ C) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0;
    for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * len + e];
    int i = (int)(e / d2), j = (int)(e % d2);
    if (i == j) s += diag_add;
    C[e] = s;
  }
}

// Double-float multiply-add (inputs split into FP32 pairs hi + lo; products
// hi*hi formed exactly as an FP32 pair with fma, the cross terms hi*lo +
// lo*hi added to the compensation; sums kept as FP32 pairs with TwoSum).  About 2^-44 relative accuracy per term at FP32 instruction rates:
// GB300 executes FP64 at ~1/60 of its FP32 rate.
__device__ __forceinline__ void df_acc(float& S, float& Cc, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  const float e = fmaf(ah, bh, -p);
  const float t = S + p;
  const float bp = t - S;
  const float err = (S - (t - bp)) + (p - bp);
  S = t;
  Cc += err + e + fmaf(ah, bl, al * bh);
}

// The same double-float Gram from inputs already split into float pairs
// (A = Ah + Al, B = Bh + Bl, row-major with leading dimensions lda, ldb):
// the tile loads are plain float loads, batched, with no FP64 conversions.
// tri: A and B lower triangular (A[q][i] = 0 for i > q), so rows
// q < max(i0, j0) contribute nothing to a tile.
__global__ void __launch_bounds__(256)
gram_dfs_kernel(const float* __restrict__ Ahg, const float* __restrict__ Alg, int64_t lda, const float* __restrict__ Bhg,
                const float* __restrict__ Blg, int64_t ldb, int64_t m, int d1, int d2, int64_t kchunk,
                double* __restrict__ part, int tri, int sym) {
  __shared__ float Ah[kGK][kGT], Al[kGK][kGT], Bh[kGK][kGT], Bl[kGK][kGT];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  int i0, j0;
  if (sym) {
    // A == B: only the tiles on and below the diagonal, blockIdx.x = ti (ti + 1) / 2 + tj
    const int t = blockIdx.x;
    int ti = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while (ti * (ti + 1) / 2 > t) --ti;
    i0 = ti * kGT;
    j0 = (t - ti * (ti + 1) / 2) * kGT;
  } else {
    i0 = blockIdx.y * kGT;
    j0 = blockIdx.x * kGT;
  }
  const int64_t k1 = min(m, (int64_t)blockIdx.z * kchunk + kchunk);
  const int64_t k0 = tri ? max((int64_t)blockIdx.z * kchunk, (int64_t)max(i0, j0)) : (int64_t)blockIdx.z * kchunk;
  float S[4][4] = {}, Cc[4][4] = {};
  for (int64_t kk = k0; kk < k1; kk += kGK) {
    float v[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u, r = e / kGT, c = e % kGT;
      const int64_t row = kk + r;
      const bool ia = row < k1 && i0 + c < d1, ib = row < k1 && j0 + c < d2;
      v[u][0] = ia ? Ahg[row * lda + i0 + c] : 0.f;
      v[u][1] = ia ? Alg[row * lda + i0 + c] : 0.f;
      v[u][2] = ib ? Bhg[row * ldb + j0 + c] : 0.f;
      v[u][3] = ib ? Blg[row * ldb + j0 + c] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u, r = e / kGT, c = e % kGT;
      Ah[r][c] = v[u][0];
      Al[r][c] = v[u][1];
      Bh[r][c] = v[u][2];
      Bl[r][c] = v[u][3];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kGK; ++r) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ah[u] = Ah[r][ty + 16 * u];
        al[u] = Al[r][ty + 16 * u];
        bh[u] = Bh[r][tx + 16 * u];
        bl[u] = Bl[r][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) df_acc(S[u][w], Cc[u][w], ah[u], al[u], bh[w], bl[w]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * w;
      if (i < d1 && j < d2) part[((int64_t)blockIdx.z * d1 + i) * d2 + j] = (double)S[u][w] + (double)Cc[u][w];
    }
}

int gram_df_split(const float* Ah, const float* Al, int64_t lda, const float* Bh, const float* Bl, int64_t ldb,
                  int64_t m, int d1, int d2, double* C, double diag_add, double* ws, int64_t ws_len, cudaStream_t st,
                  bool tri) {
  // the same operand on both sides: a symmetric result, formed from the
  // tiles on and below the diagonal only
  const bool sym = Ah == Bh && Al == Bl && lda == ldb && d1 == d2;
  const int td = ceil_div(d1, kGT);
  const int tiles = sym ? td * (td + 1) / 2 : ceil_div(d1, kGT) * ceil_div(d2, kGT);
  int ks = std::max(1, std::min<int>(ceil_div(tri ? 2 * 304 : 304, tiles), ceil_div(m, 64)));
  const int64_t len = (int64_t)d1 * d2;
  while (ks > 1 && (int64_t)ks * len > ws_len) --ks;
  if ((int64_t)ks * len > ws_len) {
    set_last_error("gram_df_split: workspace too small");
    return GBCCA_ERR_INVALID_ARG;
  }
  const int64_t kchunk = (m + ks - 1) / ks;
  dim3 grid = sym ? dim3(tiles, 1, ks) : dim3(ceil_div(d2, kGT), ceil_div(d1, kGT), ks);
  gram_dfs_kernel<<<grid, 256, 0, st>>>(Ah, Al, lda, Bh, Bl, ldb, m, d1, d2, kchunk, ws, tri ? 1 : 0, sym ? 1 : 0);
  GB_CHECK_LAUNCH();
  if (sym)
    sum_parts_sym_kernel<<<ceil_div(len, 256), 256, 0, st>>>(ws, ks, d1, diag_add, C);
  else
    sum_parts_kernel<<<ceil_div(len, 256), 256, 0, st>>>(ws, ks, len, d1, d2, diag_add, C);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

int gram_tn(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t m, int d1, int d2, double* C,
            double diag_add, double* ws, int64_t ws_len, cudaStream_t st) {
  int tiles = ceil_div(d1, kGT) * ceil_div(d2, kGT);
  int ks = std::max(1, std::min<int>(ceil_div(304, tiles), ceil_div(m, 64)));
  int64_t len = (int64_t)d1 * d2;
  while (ks > 1 && (int64_t)ks * len > ws_len) --ks;
  if ((int64_t)ks * len > ws_len) {
    set_last_error("gram_tn: workspace too small");
    return GBCCA_ERR_INVALID_ARG;
  }
  int64_t kchunk = (m + ks - 1) / ks;
  dim3 grid(ceil_div(d2, kGT), ceil_div(d1, kGT), ks);
  gram_tn_kernel<<<grid, 256, 0, st>>>(A, lda, B, ldb, m, d1, d2, kchunk, ws);
  GB_CHECK_LAUNCH();
  sum_parts_kernel<<<ceil_div(len, 256), 256, 0, st>>>(ws, ks, len, d1, d2, diag_add, C);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

// ------------------------------------------- M^{-1} in double-float form
// For FP32/BF16 plans the solver applies M^{-1} = R^{-1} R^{-T} (Table 1's
// preconditioned gradient) through an explicit symmetric matrix held as a
// float pair hi + lo (~2^-44 relative), formed once per preconditioner, and
// multiplied with double-float arithmetic.  One launch covers both views and
// replaces two dependent triangular products per view; its rounding error is
// ~2^-44 sqrt(d) kappa(M), below that of FP32 triangular products
// (~2^-24 kappa(R) each).
__global__ void split_df_kernel(const double* __restrict__ A, int64_t len, float* __restrict__ hi,
                                float* __restrict__ lo) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= len) return;
  const double x = A[e];
  const float h = (float)x;
  hi[e] = h;
  lo[e] = (float)(x - (double)h);
}

int minv_df_build(const double* Rinv, int d, float* hi, float* lo, double* ws, int64_t ws_len, cudaStream_t st) {
  const int64_t dd = (int64_t)d * d;
  if (ws_len < 5 * dd) {
    set_last_error("minv_df_build: workspace too small");
    return GBCCA_ERR_INVALID_ARG;
  }
  // T = R^{-T} (lower triangular) as a float pair, then C = T^T T = R^{-1} R^{-T}
  float* Th = reinterpret_cast<float*>(ws);
  float* Tl = Th + dd;
  double* C = ws + dd;
  GB_TRY(split_df(Rinv, d, d, true, Th, Tl, st));
  GB_TRY(gram_df_split(Th, Tl, d, Th, Tl, d, d, d, d, C, 0.0, ws + 2 * dd, ws_len - 2 * dd, st, true));
  split_df_kernel<<<ceil_div(dd, 256), 256, 0, st>>>(C, dd, hi, lo);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

__device__ __forceinline__ void df_add(float& S, float& Cc, float s2, float c2) {
  const float t = S + s2;
  const float bp = t - S;
  const float err = (S - (t - bp)) + (s2 - bp);
  S = t;
  Cc += err + c2;
}

constexpr int kMvRows = 4;            // output rows per CTA
constexpr int kMvThreads = 256;
constexpr int kMvStageBytes = 98304;  // shared memory of one staged K chunk (A rows + X rows)

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Y_b (m x c) = A_b X_b for problem b = blockIdx.y, A_b (m x K, row-major)
// and X_b (K x c, row stride ldx) as double-float pairs hi + lo.  A CTA owns
// kMvRows rows of Y.  The K range is walked in chunks: the chunk's rows of A
// and of X are copied into shared memory as (hi, lo) pairs by asynchronous
// copies (all of them in flight at once), then thread t computes output
// e = t mod (kMvRows c) over the inner indices q = t / (kMvRows c) + j KS of
// the chunk (KS = the threads per output), in two double-float chains.  The
// KS partial pairs of an output are added in fixed order through shared
// memory at the end: no scratch in global memory, no atomics, and the result
// does not depend on scheduling.
__global__ void __launch_bounds__(kMvThreads) dfmv_kernel(DfmvArgs a) {
  if (a.done != nullptr && *a.done) return;
  // the problem's fields by selection (a dynamic index into the parameter
  // array would copy it to local memory)
  const bool b1 = blockIdx.y != 0;
#define GB_SEL(f) (b1 ? a.p[1].f : a.p[0].f)
  struct {
    const float *hi, *lo, *Xh, *Xl;
    double* Y;
    int m, K, ldx, ldy;
  } P{GB_SEL(hi), GB_SEL(lo), GB_SEL(Xh), GB_SEL(Xl), GB_SEL(Y), GB_SEL(m), GB_SEL(K), GB_SEL(ldx), GB_SEL(ldy)};
#undef GB_SEL
  const int r0 = blockIdx.x * kMvRows;
  if (r0 >= P.m) return;  // uniform over the CTA
  extern __shared__ float2 mv[];
  const int c = a.c, Kc = a.kc;
  float2* As = mv;                 // [kMvRows][Kc]
  float2* Xs = mv + kMvRows * Kc;  // [Kc][c]
  const int t = threadIdx.x;
  const int nout = kMvRows * c;
  const int KS = max(1, kMvThreads / nout);
  const bool active = t < nout * KS;
  const int e = t % nout, ks = t / nout;
  const int rr = e / c, col = e - rr * c;
  float S0 = 0.f, C0 = 0.f, S1 = 0.f, C1 = 0.f;
  for (int k0 = 0; k0 < P.K; k0 += Kc) {
    const int kn = min(Kc, P.K - k0);
    __syncthreads();  // the previous chunk has been consumed
    for (int i = t; i < kMvRows * kn; i += kMvThreads) {
      const int r2 = i / kn, q = i - r2 * kn;
      float2* d = As + r2 * Kc + q;
      if (r0 + r2 < P.m) {
        const int64_t o = (int64_t)(r0 + r2) * P.K + k0 + q;
        cp_async4(&d->x, P.hi + o);
        cp_async4(&d->y, P.lo + o);
      } else {
        *d = make_float2(0.f, 0.f);
      }
    }
    for (int i = t; i < kn * c; i += kMvThreads) {
      const int q = i / c, cc = i - q * c;
      const int64_t o = (int64_t)(k0 + q) * P.ldx + cc;
      cp_async4(&Xs[i].x, P.Xh + o);
      cp_async4(&Xs[i].y, P.Xl + o);
    }
    cp_async_wait_all();
    __syncthreads();
    if (active) {
      const float2* ar = As + rr * Kc;
      int q = ks;
      for (; q + KS < kn; q += 2 * KS) {
        const float2 a0 = ar[q], x0 = Xs[q * c + col];
        const float2 a1 = ar[q + KS], x1 = Xs[(q + KS) * c + col];
        df_acc(S0, C0, a0.x, a0.y, x0.x, x0.y);
        df_acc(S1, C1, a1.x, a1.y, x1.x, x1.y);
      }
      if (q < kn) {
        const float2 a0 = ar[q], x0 = Xs[q * c + col];
        df_acc(S0, C0, a0.x, a0.y, x0.x, x0.y);
      }
    }
  }
  df_add(S0, C0, S1, C1);
  __syncthreads();
  float2* red = mv;  // [KS][nout]
  if (active) red[ks * nout + e] = make_float2(S0, C0);
  __syncthreads();
  if (t < nout && r0 + rr < P.m) {
    float s = 0.f, cc = 0.f;
    for (int k2 = 0; k2 < KS; ++k2) df_add(s, cc, red[k2 * nout + t].x, red[k2 * nout + t].y);
    P.Y[(int64_t)(r0 + rr) * P.ldy + col] = (double)s + (double)cc;
  }
}

int dfmv(const DfmvArgs& a, int nprob, cudaStream_t st) {
  if (a.c < 1 || kMvRows * a.c > kMvThreads || nprob < 1 || nprob > 2) {
    set_last_error("dfmv: unsupported column count");
    return GBCCA_ERR_INVALID_ARG;
  }
  int mmax = 0, kmax = 0;
  for (int b = 0; b < nprob; ++b) {
    if (a.p[b].ldx < a.c) {
      set_last_error("dfmv: X rows must hold c columns");
      return GBCCA_ERR_INVALID_ARG;
    }
    mmax = std::max(mmax, a.p[b].m);
    kmax = std::max(kmax, a.p[b].K);
  }
  // K chunk: the chunk's rows of A and of X (float pairs) fill at most
  // kMvStageBytes of shared memory; the final reduction reuses the space
  DfmvArgs g = a;
  g.kc = std::max(1, std::min(kmax, kMvStageBytes / (8 * (kMvRows + a.c))));
  const size_t smem = std::max<size_t>(8 * (size_t)g.kc * (kMvRows + a.c), 8 * (size_t)kMvThreads);
  GB_CUDA(cudaFuncSetAttribute(dfmv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dfmv_kernel<<<dim3(ceil_div(mmax, kMvRows), nprob), kMvThreads, smem, st>>>(g);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

// hi/lo split of the first c columns of X (rows x ldx doubles) into two
// rows x c float arrays
__global__ void split_rows_kernel(const double* __restrict__ X, int rows, int c, int ldx, float* __restrict__ hi,
                                  float* __restrict__ lo) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * c) return;
  const int i = e / c, j = e - i * c;
  const double x = X[(int64_t)i * ldx + j];
  const float h = (float)x;
  hi[e] = h;
  lo[e] = (float)(x - (double)h);
}

int split_rows(const double* X, int rows, int c, int ldx, float* hi, float* lo, cudaStream_t st) {
  split_rows_kernel<<<ceil_div(rows * c, 256), 256, 0, st>>>(X, rows, c, ldx, hi, lo);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

// hi/lo split of A (r x c) or of A^T
__global__ void split_df_t_kernel(const double* __restrict__ A, int r, int c, int trans, float* __restrict__ hi,
                                  float* __restrict__ lo) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)r * c) return;
  const int i = (int)(e / c), j = (int)(e % c);
  const double x = A[e];
  const float h = (float)x;
  const int64_t o = trans ? (int64_t)j * r + i : e;
  hi[o] = h;
  lo[o] = (float)(x - (double)h);
}

int split_df(const double* A, int r, int c, bool trans, float* hi, float* lo, cudaStream_t st) {
  split_df_t_kernel<<<ceil_div((int64_t)r * c, 256), 256, 0, st>>>(A, r, c, trans ? 1 : 0, hi, lo);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

// ------------------------------------------------- allocation-free Gram
// The same split-K Gram as gram_tn (FP64 gram_tn_kernel + sum_parts_kernel),
// with its partial slabs in a fixed static device array instead of plan
// memory.  It serves callers that may not allocate device memory at all: a
// process that has reserved HBM up front in its own pool and budgets every
// byte, or one that cannot accept the device-wide synchronization that
// cudaMalloc / cudaFree may impose on all of its streams.
//
// Limit: the scratch holds kNoAllocScratch doubles (8 MiB).  A call needs at
// least one d x d partial slab, so d <= 1024; larger d is rejected with
// GBCCA_ERR_INVALID_ARG before any device work.  The number of split-K slabs
// is as many as fit (up to one per 64 rows and enough CTAs for the GPU).  Nothing in the scratch has
// to start at zero: every element of a slab that the second kernel reads is
// written by the first.  The scratch is one buffer per device shared by all
// callers, so two calls whose kernels may overlap in time (different streams,
// or threads without ordering) race on it; callers order them.
constexpr int64_t kNoAllocScratch = int64_t(1) << 20;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch for the current device, looked up once per
// device.  The first call on a device resolves the symbol (which can load the
// module), so a caller that records work into a stream capture makes one
// call on that device before capturing.
int noalloc_scratch(double** out) {
  int dev = -1;
  GB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_last_error("allocation-free Gram: device ordinal out of range");
    return GBCCA_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_last_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      return GBCCA_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return GBCCA_OK;
}
}  // namespace

int noalloc_max_d() {
  int d = 1;
  while ((int64_t)(d + 1) * (d + 1) <= kNoAllocScratch) ++d;
  return d;
}

int gram_noalloc(const double* A, int64_t lda, int64_t m, int d, double lambda, double* C, cudaStream_t st) {
  const int64_t len = (int64_t)d * d;
  if (len > kNoAllocScratch) {
    set_last_error("allocation-free Gram: d = " + std::to_string(d) + " exceeds the " +
                   std::to_string(noalloc_max_d()) + " columns its 8 MiB static scratch holds");
    return GBCCA_ERR_INVALID_ARG;
  }
  double* ws = nullptr;
  GB_TRY(noalloc_scratch(&ws));
  const int tiles = ceil_div(d, kGT) * ceil_div(d, kGT);
  int ks = std::max(1, std::min<int>(ceil_div(304, tiles), ceil_div(m, 64)));
  while (ks > 1 && (int64_t)ks * len > kNoAllocScratch) --ks;
  const int64_t kchunk = (m + ks - 1) / ks;
  dim3 grid(ceil_div(d, kGT), ceil_div(d, kGT), ks);
  gram_tn_kernel<<<grid, 256, 0, st>>>(A, lda, A, lda, m, d, d, kchunk, ws);
  GB_CHECK_LAUNCH();
  sum_parts_kernel<<<ceil_div(len, 256), 256, 0, st>>>(ws, ks, len, d, d, lambda, C);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

// --------------------------------------------------------------- Cholesky
// Right-looking blocked Cholesky of a symmetric positive definite d x d
// matrix (only its lower triangle is read): A = L L^T with 32 x 32 blocks.
// At the end R = L^T is written to the upper triangle and the strict lower
// triangle is zeroed, so A holds R with R^T R = A.  A non-positive pivot sets
// *flag = 1 (the caller reports GBCCA_ERR_NOT_SPD).
constexpr int kNB = 32;

__global__ void __launch_bounds__(128) chol_diag_kernel(double* A, int d, int p, int* flag) {
  // The 32 x 32 diagonal block in shared memory, factored by 4 warps: GB300
  // issues FP64 at a small fraction of its FP32 rate on each of the SM's four
  // schedulers, so the trailing updates of every step are spread over all four.
  __shared__ double L[kNB][kNB + 1];
  __shared__ double s_r;
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  const int o = p * kNB, nb = min(kNB, d - o);
  for (int e = tid; e < kNB * kNB; e += blockDim.x) {
    const int r = e / kNB, c = e % kNB;
    L[r][c] = (r < nb && c <= r) ? A[(int64_t)(o + r) * d + o + c] : 0.0;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      double piv = L[j][j];
      if (!(piv > 0.0)) {
        s_bad = 1;
        piv = 1.0;  // keep going with a harmless value; the result is discarded
      }
      const double rj = rsqrt_nr(piv);
      L[j][j] = piv * rj;
      s_r = rj;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < nb; i += blockDim.x) L[i][j] *= s_r;
    __syncthreads();
    // trailing lower triangle (i, c), j < c <= i < nb, enumerated row by row
    const int m = nb - j - 1, cnt = m * (m + 1) / 2;
    for (int e = tid; e < cnt; e += blockDim.x) {
      int i1 = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
      while ((i1 + 1) * (i1 + 2) / 2 <= e) ++i1;
      while (i1 * (i1 + 1) / 2 > e) --i1;
      const int i = j + 1 + i1, c = j + 1 + (e - i1 * (i1 + 1) / 2);
      L[i][c] -= L[i][j] * L[c][j];
    }
    __syncthreads();
  }
  if (tid == 0 && s_bad) atomicExch(flag, kFlagNotSpd);
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    if (c <= r) A[(int64_t)(o + r) * d + o + c] = L[r][c];
  }
}

// A[i-block, p] <- A[i-block, p] L_pp^{-T}: one warp per row, lane c holding
// x_c; forward substitution in column order, each solved x_c broadcast by a
// shuffle to the lanes that still subtract it (the same multiply-adds, in the
// same order, as a serial substitution of the row).
constexpr int kTrsmRows = 8;  // rows (warps) per CTA
__global__ void __launch_bounds__(32 * kTrsmRows) chol_trsm_kernel(double* A, int d, int p) {
  __shared__ double L[kNB][kNB + 1];
  __shared__ double rinv[kNB];
  const int o = p * kNB, nb = min(kNB, d - o);
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    int r = e / kNB, c = e % kNB;
    L[r][c] = (r < nb && c <= r) ? A[(int64_t)(o + r) * d + o + c] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < kNB) rinv[threadIdx.x] = threadIdx.x < nb ? 1.0 / L[threadIdx.x][threadIdx.x] : 1.0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int row = o + nb + blockIdx.x * kTrsmRows + (threadIdx.x >> 5);
  if (row >= d) return;  // uniform over the warp
  double acc = lane < nb ? A[(int64_t)row * d + o + lane] : 0.0;
  double x = 0.0;
  for (int c = 0; c < nb; ++c) {
    if (lane == c) x = acc * rinv[c];
    const double xc = __shfl_sync(0xffffffffu, x, c);
    if (lane > c) acc -= L[lane][c] * xc;
  }
  if (lane < nb) A[(int64_t)row * d + o + lane] = x;
}

// trailing update A[I, J] -= A[I, p] A[J, p]^T for block pairs I >= J > p.
__global__ void chol_syrk_kernel(double* A, int d, int p) {
  const int o = p * kNB, nb = min(kNB, d - o);
  int I = blockIdx.y + p + 1, J = blockIdx.x + p + 1;
  if (J > I) return;
  __shared__ double a[kNB][kNB + 1], b[kNB][kNB + 1];
  const int i0 = I * kNB, j0 = J * kNB;
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    int r = e / kNB, c = e % kNB;
    a[r][c] = (i0 + r < d && c < nb) ? A[(int64_t)(i0 + r) * d + o + c] : 0.0;
    b[r][c] = (j0 + r < d && c < nb) ? A[(int64_t)(j0 + r) * d + o + c] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    int r = e / kNB, c = e % kNB;
    int i = i0 + r, j = j0 + c;
    if (i >= d || j >= d || j > i) continue;
    double s = 0;
#pragma unroll 8
    for (int q = 0; q < kNB; ++q) s += a[r][q] * b[c][q];
    A[(int64_t)i * d + j] -= s;
  }
}

__global__ void lower_to_upper_kernel(double* A, int d) {
  int i = blockIdx.y * 32 + threadIdx.y, j = blockIdx.x * 32 + threadIdx.x;
  if (i >= d || j >= d || j < i) return;
  double l = A[(int64_t)j * d + i];  // L[j][i], j >= i
  A[(int64_t)i * d + j] = l;          // R[i][j]
  if (j > i) A[(int64_t)j * d + i] = 0.0;
}

int cholesky_upper(double* A, int d, int* flag, cudaStream_t st) {
  int nbk = ceil_div(d, kNB);
  for (int p = 0; p < nbk; ++p) {
    chol_diag_kernel<<<1, 128, 0, st>>>(A, d, p, flag);
    GB_CHECK_LAUNCH();
    int below = d - (p + 1) * kNB;
    if (below > 0) {
      chol_trsm_kernel<<<ceil_div(below, kTrsmRows), 32 * kTrsmRows, 0, st>>>(A, d, p);
      GB_CHECK_LAUNCH();
      int nt = nbk - p - 1;
      chol_syrk_kernel<<<dim3(nt, nt), 256, 0, st>>>(A, d, p);
      GB_CHECK_LAUNCH();
    }
  }
  lower_to_upper_kernel<<<dim3(ceil_div(d, 32), ceil_div(d, 32)), dim3(32, 32), 0, st>>>(A, d);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

// ------------------------------------------------------- triangular inverse
// Rinv = R^{-1} for upper-triangular R by recursive doubling over aligned
// diagonal blocks: the 32 x 32 diagonal blocks are inverted by back
// substitution, then at each level h = 32, 64, ... the inverted neighbours
// A = [r0, r0+h) and C = [c0, c1) (c0 = r0 + h) are joined through
//   Rinv[A, C] = -Rinv[A, A] (R[A, C] Rinv[C, C]),
// two FP64 products per level.  Every level is one parallel launch pair, so
// the d^3/3 multiply-adds spread over all SMs.
constexpr int kTB = 32;

__global__ void tri_diag_inv_kernel(const double* __restrict__ R, double* __restrict__ Rinv, int d) {
  __shared__ double L[kTB][kTB + 1];
  __shared__ double X[kTB][kTB + 1];
  __shared__ double rinv[kTB];
  const int o = blockIdx.x * kTB, nb = min(kTB, d - o), j = threadIdx.x;
  for (int r = 0; r < kTB; ++r) L[r][j] = (r < nb && j < nb && j >= r) ? R[(int64_t)(o + r) * d + o + j] : 0.0;
  __syncthreads();
  rinv[j] = j < nb ? 1.0 / L[j][j] : 0.0;
  __syncthreads();
  for (int i = kTB - 1; i >= 0; --i) {
    double x = 0.0;
    if (i <= j && j < nb) {
      double s = 0.0;
      for (int q = i + 1; q <= j; ++q) s += L[i][q] * X[q][j];
      x = ((i == j) ? 1.0 : 0.0) - s;
      x *= rinv[i];
    }
    X[i][j] = x;  // each thread owns column j: no barrier needed
  }
  for (int r = 0; r < nb; ++r)
    if (j < nb) Rinv[(int64_t)(o + r) * d + o + j] = X[r][j];
}

// stage 0: T_p = R[A, C] Rinv[C, C]  (h x w, row stride h)
// stage 1: Rinv[A, C] = -Rinv[A, A] T_p
// Grid (ceil(h/32), ceil(h/32), pairs); each CTA one 32 x 32 output tile,
// K in chunks of 32 restricted to where the triangular factor is non-zero.
template <int kStage>
__global__ void __launch_bounds__(256) tri_level_kernel(const double* __restrict__ R, double* __restrict__ Rinv,
                                                        double* __restrict__ T, int d, int h) {
  __shared__ double As[kTB][kTB + 1], Bs[kTB][kTB + 1];
  const int p = blockIdx.z;
  const int r0 = 2 * p * h, c0 = r0 + h;
  if (c0 >= d) return;
  const int w = min(d, c0 + h) - c0;
  const int i0 = blockIdx.y * kTB, j0 = blockIdx.x * kTB;
  if (i0 >= h || j0 >= w) return;
  double* Tp = T + (int64_t)p * h * h;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  // K range: stage 0 runs q in [0, w) with Rinv[C,C][q][j] = 0 for q > j;
  // stage 1 runs q in [0, h) with Rinv[A,A][i][q] = 0 for q < i
  const int klo = kStage == 0 ? 0 : i0;
  const int khi = kStage == 0 ? min(w, j0 + kTB) : h;
  double acc[2][2] = {};
  for (int k0 = klo; k0 < khi; k0 += kTB) {
    for (int e = threadIdx.x; e < kTB * kTB; e += 256) {
      const int r = e / kTB, c = e % kTB;
      const int ia = i0 + r, qa = k0 + c;  // A tile element (i, q)
      const int qb = k0 + r, jb = j0 + c;  // B tile element (q, j)
      double av = 0.0, bv = 0.0;
      if (kStage == 0) {
        if (ia < h && qa < khi) av = R[(int64_t)(r0 + ia) * d + c0 + qa];
        if (qb < khi && jb < w) bv = Rinv[(int64_t)(c0 + qb) * d + c0 + jb];
      } else {
        if (ia < h && qa < khi) av = Rinv[(int64_t)(r0 + ia) * d + r0 + qa];
        if (qb < khi && jb < w) bv = Tp[(int64_t)qb * h + jb];
      }
      As[r][c] = av;
      Bs[r][c] = bv;
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < kTB; ++q) {
      const double a0 = As[ty][q], a1 = As[ty + 16][q];
      const double b0 = Bs[q][tx], b1 = Bs[q][tx + 16];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < h && j < w) {
        if (kStage == 0)
          Tp[(int64_t)i * h + j] = acc[u][v];
        else
          Rinv[(int64_t)(r0 + i) * d + c0 + j] = -acc[u][v];
      }
    }
}

int tri_inverse_upper(const double* R, double* Rinv, int d, double* ws, int64_t ws_len, cudaStream_t st) {
  if (ws_len < (int64_t)d * d) {
    set_last_error("tri_inverse_upper: workspace too small");
    return GBCCA_ERR_INVALID_ARG;
  }
  GB_CUDA(cudaMemsetAsync(Rinv, 0, sizeof(double) * d * d, st));
  tri_diag_inv_kernel<<<ceil_div(d, kTB), kTB, 0, st>>>(R, Rinv, d);
  GB_CHECK_LAUNCH();
  for (int h = kTB; h < d; h *= 2) {
    const int pairs = ceil_div(d - h, 2 * h);
    dim3 grid(ceil_div(h, kTB), ceil_div(h, kTB), pairs);
    tri_level_kernel<0><<<grid, 256, 0, st>>>(R, Rinv, ws, d, h);
    GB_CHECK_LAUNCH();
    tri_level_kernel<1><<<grid, 256, 0, st>>>(R, Rinv, ws, d, h);
    GB_CHECK_LAUNCH();
  }
  return GBCCA_OK;
}

__global__ void to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t len) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

int to_f32(const double* a, float* b, int64_t len, cudaStream_t st) {
  to_f32_kernel<<<std::min(ceil_div(len, 256), 4096), 256, 0, st>>>(a, b, len);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

// ------------------------------------------------------ factor x thin block
// C (m x c) = op(A) B with A ra x ca row-major (op = identity or transpose),
// B (rows = columns of op(A)) and C FP64 with row strides ldb, ldc.  T = double
// (FP64 path) or float (the FP32 copy of R^{-1} used with BF16/FP32 data).
// With tri set, A is upper triangular and its zero tiles are skipped.
// Grid = (16-row blocks) x (64-wide slices of the inner dimension); each CTA
// writes a partial product and a second kernel adds the slices in order.
constexpr int kMR = 16, kMK = 64, kMC = 40;

template <typename T>
__global__ void __launch_bounds__(128)
mat_thin_kernel(const T* __restrict__ A, int ra, int ca, int transA, int tri, const double* __restrict__ B,
                int64_t ldb, double* __restrict__ part, int c) {
  __shared__ T As[kMK][kMR + 1];   // As[l][r] = op(A)[i0 + r][l0 + l]
  __shared__ T Bs[kMK][kMC];
  const int tr = threadIdx.x & 15, tg = threadIdx.x >> 4;  // row, column group (8 groups)
  const int m = transA ? ca : ra;   // rows of op(A)
  const int K = transA ? ra : ca;   // columns of op(A)
  const int i0 = blockIdx.x * kMR, l0 = blockIdx.y * kMK;
  double* out = part + ((int64_t)blockIdx.y * m) * c;
  // op(A)[i][l] is nonzero only for l >= i (A upper) or l <= i (A^T lower)
  const bool zero = (tri && !transA && l0 + kMK - 1 < i0) || (tri && transA && l0 > i0 + kMR - 1);
  T acc[kMC / 8] = {};
  if (!zero) {
    if (transA) {
      for (int e = threadIdx.x; e < kMK * kMR; e += 128) {
        int l = e / kMR, r = e % kMR;
        As[l][r] = (l0 + l < K && i0 + r < m) ? A[(int64_t)(l0 + l) * ca + i0 + r] : T(0);
      }
    } else {
      for (int e = threadIdx.x; e < kMK * kMR; e += 128) {
        int r = e / kMK, l = e % kMK;
        As[l][r] = (l0 + l < K && i0 + r < m) ? A[(int64_t)(i0 + r) * ca + l0 + l] : T(0);
      }
    }
    for (int e = threadIdx.x; e < kMK * kMC; e += 128) {
      int l = e / kMC, cc = e % kMC;
      Bs[l][cc] = (l0 + l < K && cc < c) ? (T)B[(int64_t)(l0 + l) * ldb + cc] : T(0);
    }
    __syncthreads();
#pragma unroll 16
    for (int l = 0; l < kMK; ++l) {
      const T a = As[l][tr];
#pragma unroll
      for (int q = 0; q < kMC / 8; ++q) acc[q] += a * Bs[l][tg + 8 * q];
    }
  }
  const int i = i0 + tr;
  if (i < m) {
#pragma unroll
    for (int q = 0; q < kMC / 8; ++q) {
      const int cc = tg + 8 * q;
      if (cc < c) out[(int64_t)i * c + cc] = (double)acc[q];
    }
  }
}

__global__ void mat_thin_sum_kernel(const double* __restrict__ part, int nslices, int m, int c,
                                    double* __restrict__ C, int64_t ldc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * c) return;
  double s = 0;
  for (int q = 0; q < nslices; ++q) s += part[(int64_t)q * m * c + e];
  C[(int64_t)(e / c) * ldc + e % c] = s;
}

template <typename T>
int mat_thin(const T* A, int ra, int ca, bool transA, bool tri, const double* B, int64_t ldb, double* C,
             int64_t ldc, int c, double* part, cudaStream_t st) {
  const int m = transA ? ca : ra;
  const int K = transA ? ra : ca;
  const int ns = ceil_div(K, kMK);
  for (int c0 = 0; c0 < c; c0 += kMC) {
    const int cw = std::min(kMC, c - c0);
    mat_thin_kernel<T><<<dim3(ceil_div(m, kMR), ns), 128, 0, st>>>(A, ra, ca, transA ? 1 : 0, tri ? 1 : 0, B + c0,
                                                                   ldb, part, cw);
    GB_CHECK_LAUNCH();
    mat_thin_sum_kernel<<<ceil_div(m * cw, 256), 256, 0, st>>>(part, ns, m, cw, C + c0, ldc);
    GB_CHECK_LAUNCH();
  }
  return GBCCA_OK;
}
template int mat_thin<double>(const double*, int, int, bool, bool, const double*, int64_t, double*, int64_t, int,
                              double*, cudaStream_t);
template int mat_thin<float>(const float*, int, int, bool, bool, const double*, int64_t, double*, int64_t, int,
                             double*, cudaStream_t);

}  // namespace gbcca
