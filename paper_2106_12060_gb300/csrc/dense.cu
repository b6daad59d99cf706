// Small dense FP64 linear algebra for the preconditioner (Sec. 3): the Gram of
// the sketch, its Cholesky factor R (R^T R = (S Z)^T (S Z) + lambda I, the R
// of the QR of [S Z; sqrt(lambda) I]), R^{-1}, and products of d x d factors
// with d x c blocks (the M^{-1} = R^{-1} R^{-T} applications of Table 1).
//
// GB300 executes FP64 at ~1/60 of its FP32 rate, so these kernels spread the
// O(s d^2) and O(d^3) work over many CTAs (split-K Gram, blocked right-looking
// Cholesky, one warp per column of R^{-1}).
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

// --------------------------------------------------------------- Cholesky
// Right-looking blocked Cholesky of a symmetric positive definite d x d
// matrix (only its lower triangle is read): A = L L^T with 32 x 32 blocks.
// At the end R = L^T is written to the upper triangle and the strict lower
// triangle is zeroed, so A holds R with R^T R = A.  A non-positive pivot sets
// *flag = 1 (the caller reports GBCCA_ERR_NOT_SPD).
constexpr int kNB = 32;

__global__ void chol_diag_kernel(double* A, int d, int p, int* flag) {
  __shared__ double a[kNB][kNB + 1];
  const int lane = threadIdx.x;
  const int o = p * kNB, nb = min(kNB, d - o);
  for (int c = 0; c < nb; ++c) a[lane][c] = lane < nb ? A[(int64_t)(o + lane) * d + o + c] : 0.0;
  __syncwarp();
  for (int j = 0; j < nb; ++j) {
    double piv = a[j][j];
    if (piv <= 0.0 || !(piv == piv)) {
      if (lane == 0) atomicExch(flag, 1);
      piv = 1.0;  // keep going with a harmless value; the result is discarded
    }
    double ljj = sqrt(piv);
    __syncwarp();
    if (lane == j) a[j][j] = ljj;
    if (lane > j && lane < nb) a[lane][j] /= ljj;
    __syncwarp();
    if (lane > j && lane < nb)
      for (int c = j + 1; c <= lane; ++c) a[lane][c] -= a[lane][j] * a[c][j];
    __syncwarp();
  }
  if (lane < nb)
    for (int c = 0; c <= lane; ++c) A[(int64_t)(o + lane) * d + o + c] = a[lane][c];
}

// A[i-block, p] <- A[i-block, p] L_pp^{-T}: each thread solves one row by
// forward substitution with L_pp.
__global__ void chol_trsm_kernel(double* A, int d, int p) {
  __shared__ double L[kNB][kNB + 1];
  const int o = p * kNB, nb = min(kNB, d - o);
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    int r = e / kNB, c = e % kNB;
    L[r][c] = (r < nb && c <= r) ? A[(int64_t)(o + r) * d + o + c] : 0.0;
  }
  __syncthreads();
  const int row = o + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= d) return;
  double x[kNB];
#pragma unroll
  for (int c = 0; c < kNB; ++c) x[c] = c < nb ? A[(int64_t)row * d + o + c] : 0.0;
#pragma unroll
  for (int c = 0; c < kNB; ++c) {
    if (c < nb) {
      double s = x[c];
#pragma unroll
      for (int q = 0; q < c; ++q) s -= L[c][q] * x[q];
      x[c] = s / L[c][c];
    }
  }
#pragma unroll
  for (int c = 0; c < kNB; ++c)
    if (c < nb) A[(int64_t)row * d + o + c] = x[c];
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
    chol_diag_kernel<<<1, 32, 0, st>>>(A, d, p, flag);
    GB_CHECK_LAUNCH();
    int below = d - (p + 1) * kNB;
    if (below > 0) {
      chol_trsm_kernel<<<ceil_div(below, 64), 64, 0, st>>>(A, d, p);
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
// Rinv = R^{-1} for upper-triangular R: column j solves R x = e_j by back
// substitution; one warp per column, the inner products split over lanes.
__global__ void tri_inv_kernel(const double* __restrict__ R, double* __restrict__ Rinv, int d) {
  extern __shared__ double xs[];  // [8][d]
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + w;
  if (j >= d) return;
  double* x = xs + (int64_t)w * d;
  for (int i = lane; i < d; i += 32) x[i] = 0.0;
  __syncwarp();
  for (int i = j; i >= 0; --i) {
    double s = 0;
    for (int q = i + 1 + lane; q <= j; q += 32) s += R[(int64_t)i * d + q] * x[q];
    s = warp_sum(s);
    if (lane == 0) x[i] = ((i == j ? 1.0 : 0.0) - s) / R[(int64_t)i * d + i];
    __syncwarp();
  }
  for (int i = lane; i < d; i += 32) Rinv[(int64_t)i * d + j] = x[i];
}

int tri_inverse_upper(const double* R, double* Rinv, int d, cudaStream_t st) {
  size_t smem = sizeof(double) * 8 * d;
  GB_CUDA(cudaFuncSetAttribute(tri_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  tri_inv_kernel<<<ceil_div(d, 8), 256, smem, st>>>(R, Rinv, d);
  GB_CHECK_LAUNCH();
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
