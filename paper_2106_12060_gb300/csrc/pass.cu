// The per-iteration data pass on CUDA cores (any storage type) and the LDA
// class statistics.
//
// One Riemannian-CG iteration needs, for Phi_x = [U, eta_U], Phi_y = [V, eta_V]
// (Sec. 4.2 gradient, Table 1 retraction and projection, Cor. 4.6 cost):
//   W = [X Phi_x, Y Phi_y] (n x 4k),  Z^T W for Z = [X | Y],  W^T W.
// For FDA (Sec. 5.1-5.2) with Phi = [W, eta]: P = Xhat Phi with Xhat the
// class-centred data, Xhat^T P = S_w Phi and P^T P.
//
// Kernel A forms W row tile by row tile (and its Gram, and for FDA subtracts
// the class-mean rows and accumulates per-class column sums of P); kernel B
// accumulates Z^T W over row chunks x column blocks; a fixed-order reduction
// sums the per-CTA partials in FP64, so results are bitwise reproducible.
#include "plan.h"

namespace gbcca {

struct PassViews {
  const void* Z[2];
  int64_t ld[2];
  int d[2];
  int dofs[2];      // first row of the view in G (0, dx)
  int ocol[2];      // first column of the view's block in W
  const void* Phi[2];
  int nviews;
  int k2;           // columns of Phi used per view
  int phistride;    // row stride of Phi
  const int* done;  // skip the pass when the solver has stopped (may be null)
};

constexpr int kTM = 64;   // rows per tile in kernel A
constexpr int kTB = 32;   // rows per step in kernel B
constexpr int kGI = 25;   // Gram entries per thread (NC <= 80)
constexpr int kCI = 10;   // class-sum entries per thread (l * NC <= 2560)

template <typename Tin, typename Tacc, int RN>
__global__ void __launch_bounds__(256)
pass_w_kernel(PassViews pv, int64_t n, int NC, Tacc* __restrict__ W, double* __restrict__ partGram,
              const int32_t* __restrict__ labels, const Tacc* __restrict__ Cls, int l,
              double* __restrict__ partCls) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tacc* Zs = reinterpret_cast<Tacc*>(smem_raw);              // [32][kTM + 1]
  Tacc* Ps = Zs + 32 * (kTM + 1);                             // [32][8 * RN]
  Tacc* Wt = Ps + 32 * 8 * RN;                                // [kTM][NC]
  int* ys = reinterpret_cast<int*>(Wt + kTM * NC);            // [kTM]
  if (pv.done != nullptr && *pv.done) return;
  const int tid = threadIdx.x;
  const int tr = tid & 31, tc = tid >> 5;
  const int PW = 8 * RN;

  // per-tile sums are formed in Tacc and added into FP64 accumulators, so
  // FP32 rounding only ever acts on sums of kTM = 64 terms
  double g_acc[kGI];
#pragma unroll
  for (int i = 0; i < kGI; ++i) g_acc[i] = 0;
  double c_acc[kCI];
#pragma unroll
  for (int i = 0; i < kCI; ++i) c_acc[i] = 0;

  const int64_t ntiles = (n + kTM - 1) / kTM;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * kTM;
    for (int v = 0; v < pv.nviews; ++v) {
      const Tin* Z = reinterpret_cast<const Tin*>(pv.Z[v]);
      const Tacc* Phi = reinterpret_cast<const Tacc*>(pv.Phi[v]);
      const int d = pv.d[v];
      Tacc acc[2][RN];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int q = 0; q < RN; ++q) acc[a][q] = 0;
      for (int j0 = 0; j0 < d; j0 += 32) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          int e = tid + 256 * i;
          int r = e >> 5, c = e & 31;
          int64_t row = row0 + r;
          Tacc val = 0;
          if (row < n && j0 + c < d) val = ld_as<Tacc, Tin>(Z + row * pv.ld[v] + j0 + c);
          Zs[c * (kTM + 1) + r] = val;
        }
        for (int e = tid; e < 32 * PW; e += 256) {
          int jj = e / PW, c = e % PW;
          Tacc val = 0;
          if (j0 + jj < d && c < pv.k2) val = Phi[(int64_t)(j0 + jj) * pv.phistride + c];
          Ps[jj * PW + c] = val;
        }
        __syncthreads();
#pragma unroll 8
        for (int jj = 0; jj < 32; ++jj) {
          Tacc z0 = Zs[jj * (kTM + 1) + tr], z1 = Zs[jj * (kTM + 1) + tr + 32];
#pragma unroll
          for (int q = 0; q < RN; ++q) {
            Tacc pp = Ps[jj * PW + tc + 8 * q];
            acc[0][q] += z0 * pp;
            acc[1][q] += z1 * pp;
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int q = 0; q < RN; ++q) {
          int c = tc + 8 * q;
          if (c < pv.k2) Wt[(tr + 32 * a) * NC + pv.ocol[v] + c] = acc[a][q];
        }
    }
    if (labels != nullptr && tid < kTM) {
      int64_t row = row0 + tid;
      ys[tid] = row < n ? labels[row] : -1;
    }
    __syncthreads();
    // FDA: P = X Phi - (class mean) Phi; rows past n are zeroed.
    for (int e = tid; e < kTM * NC; e += 256) {
      int r = e / NC, c = e % NC;
      int64_t row = row0 + r;
      Tacc val = Wt[e];
      if (row >= n) val = 0;
      else if (labels != nullptr) val -= Cls[ys[r] * NC + c];
      Wt[e] = val;
      if (W != nullptr && row < n) W[row * NC + c] = val;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kGI; ++i) {
      int e = tid + 256 * i;
      if (e < NC * NC) {
        int a = e / NC, b = e % NC;
        Tacc s = 0;
        for (int r = 0; r < kTM; ++r) s += Wt[r * NC + a] * Wt[r * NC + b];
        g_acc[i] += (double)s;
      }
    }
    if (labels != nullptr) {
#pragma unroll
      for (int i = 0; i < kCI; ++i) {
        int e = tid + 256 * i;
        if (e < l * NC) {
          int cls = e / NC, c = e % NC;
          Tacc s = 0;
          for (int r = 0; r < kTM; ++r)
            if (ys[r] == cls) s += Wt[r * NC + c];
          c_acc[i] += (double)s;
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < kGI; ++i) {
    int e = tid + 256 * i;
    if (e < NC * NC) partGram[(int64_t)blockIdx.x * NC * NC + e] = g_acc[i];
  }
  if (labels != nullptr) {
#pragma unroll
    for (int i = 0; i < kCI; ++i) {
      int e = tid + 256 * i;
      if (e < l * NC) partCls[(int64_t)blockIdx.x * l * NC + e] = c_acc[i];
    }
  }
}

template <typename Tin, typename Tacc, int RQ>
__global__ void __launch_bounds__(256)
pass_g_kernel(PassViews pv, int64_t n, int NC, int D, const Tacc* __restrict__ W,
              int64_t rows_per_chunk, int nb0, double* __restrict__ partG) {
  __shared__ Tacc Zs[kTB][64];
  __shared__ Tacc Ws[kTB][8 * RQ];
  if (pv.done != nullptr && *pv.done) return;
  const int tid = threadIdx.x;
  const int tj = tid & 31, tc = tid >> 5;
  const int PW = 8 * RQ;
  const int b = blockIdx.y;
  const int v = b < nb0 ? 0 : 1;
  const int c0 = 64 * (v == 0 ? b : b - nb0);
  const int d = pv.d[v];
  const Tin* Z = reinterpret_cast<const Tin*>(pv.Z[v]);
  const int64_t r0 = blockIdx.x * rows_per_chunk;
  const int64_t r1 = min(n, r0 + rows_per_chunk);
  // Tacc partial sums over at most kFlush rows, then FP64 accumulation
  constexpr int kFlush = 4 * kTB;
  Tacc acc[2][RQ];
  double acc64[2][RQ];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int q = 0; q < RQ; ++q) acc[a][q] = 0, acc64[a][q] = 0;
  for (int64_t i0 = r0; i0 < r1; i0 += kTB) {
    if (((i0 - r0) % kFlush) == 0 && i0 != r0) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int q = 0; q < RQ; ++q) acc64[a][q] += (double)acc[a][q], acc[a][q] = 0;
    }
#pragma unroll
    for (int i = 0; i < (kTB * 64) / 256; ++i) {
      int e = tid + 256 * i;
      int r = e >> 6, c = e & 63;
      int64_t row = i0 + r;
      Tacc val = 0;
      if (row < r1 && c0 + c < d) val = ld_as<Tacc, Tin>(Z + row * pv.ld[v] + c0 + c);
      Zs[r][c] = val;
    }
    for (int e = tid; e < kTB * PW; e += 256) {
      int r = e / PW, c = e % PW;
      int64_t row = i0 + r;
      Ws[r][c] = (row < r1 && c < NC) ? W[row * NC + c] : Tacc(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int i = 0; i < kTB; ++i) {
      Tacc z0 = Zs[i][tj], z1 = Zs[i][tj + 32];
#pragma unroll
      for (int q = 0; q < RQ; ++q) {
        Tacc w = Ws[i][tc + 8 * q];
        acc[0][q] += z0 * w;
        acc[1][q] += z1 * w;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    int col = c0 + tj + 32 * a;
    if (col >= d) continue;
    int64_t grow = pv.dofs[v] + col;
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
      int c = tc + 8 * q;
      if (c < NC) partG[((int64_t)blockIdx.x * D + grow) * NC + c] = acc64[a][q] + (double)acc[a][q];
    }
  }
}

// The same product for FP32 data with the loads pipelined: each stage is a
// 32-row x 64-column block of Z (16-byte cp.async copies) and the same 32
// rows of W (4-byte copies), kGStages stages in flight, zero-filled past the
// edges.  The arithmetic (per-thread order, FP32 partial sums flushed to FP64
// every kFlush rows) is that of pass_g_kernel.  Requires d % 4 == 0,
// ld % 4 == 0 and 16-byte aligned bases (checked by the caller).
constexpr int kGStages = 4;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int RQ>
__global__ void __launch_bounds__(256)
pass_g_async_kernel(PassViews pv, int64_t n, int NC, int D, const float* __restrict__ W,
                    int64_t rows_per_chunk, int nb0, double* __restrict__ partG) {
  constexpr int PW = 8 * RQ;
  extern __shared__ __align__(16) unsigned char gsm[];
  float* Zs = reinterpret_cast<float*>(gsm);           // [kGStages][kTB][64]
  float* Ws = Zs + kGStages * kTB * 64;                 // [kGStages][kTB][PW]
  if (pv.done != nullptr && *pv.done) return;
  const int tid = threadIdx.x;
  const int tj = tid & 31, tc = tid >> 5;
  const int b = blockIdx.y;
  const int v = b < nb0 ? 0 : 1;
  const int c0 = 64 * (v == 0 ? b : b - nb0);
  const int d = pv.d[v];
  const float* Z = reinterpret_cast<const float*>(pv.Z[v]);
  const int64_t ld = pv.ld[v];
  const int64_t r0 = blockIdx.x * rows_per_chunk;
  const int64_t r1 = min(n, r0 + rows_per_chunk);
  const int nsteps = r1 > r0 ? (int)((r1 - r0 + kTB - 1) / kTB) : 0;
  // W columns NC .. PW - 1 are never copied: zero them once
  for (int e = tid; e < kGStages * kTB * PW; e += 256)
    if (e % PW >= NC) Ws[e] = 0.f;
  auto issue = [&](int step) {
    const int slot = step % kGStages;
    const int64_t i0 = r0 + (int64_t)step * kTB;
#pragma unroll
    for (int u = 0; u < (kTB * 16) / 256; ++u) {
      const int e = tid + 256 * u;  // 16-byte chunk: row e / 16, columns 4 (e % 16) ..
      const int r = e >> 4, c = 4 * (e & 15);
      const int64_t row = i0 + r;
      const bool ok = row < r1 && c0 + c < d;
      const float* src = ok ? Z + row * ld + c0 + c : Z;
      cp_async16((uint32_t)__cvta_generic_to_shared(Zs + (slot * kTB + r) * 64 + c), src, ok ? 16u : 0u);
    }
    for (int e = tid; e < kTB * NC; e += 256) {
      const int r = e / NC, c = e - r * NC;
      const int64_t row = i0 + r;
      const bool ok = row < r1;
      const float* src = ok ? W + row * NC + c : W;
      cp_async4((uint32_t)__cvta_generic_to_shared(Ws + (slot * kTB + r) * PW + c), src, ok ? 4u : 0u);
    }
  };
  constexpr int kFlush = 4 * kTB;
  float acc[2][RQ];
  double acc64[2][RQ];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int q = 0; q < RQ; ++q) acc[a][q] = 0.f, acc64[a][q] = 0.0;
#pragma unroll
  for (int s = 0; s < kGStages - 1; ++s) {
    if (s < nsteps) issue(s);
    cp_async_commit();
  }
  for (int step = 0; step < nsteps; ++step) {
    cp_async_wait<kGStages - 2>();  // this thread's copies of stage `step` have landed
    __syncthreads();                // everyone's have; the slot of step - 1 is free
    if (step + kGStages - 1 < nsteps) issue(step + kGStages - 1);
    cp_async_commit();
    if (step > 0 && (step * kTB) % kFlush == 0) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int q = 0; q < RQ; ++q) acc64[a][q] += (double)acc[a][q], acc[a][q] = 0.f;
    }
    const float* zs = Zs + (step % kGStages) * kTB * 64;
    const float* wsl = Ws + (step % kGStages) * kTB * PW;
#pragma unroll 8
    for (int i = 0; i < kTB; ++i) {
      const float z0 = zs[i * 64 + tj], z1 = zs[i * 64 + tj + 32];
#pragma unroll
      for (int q = 0; q < RQ; ++q) {
        const float w = wsl[i * PW + tc + 8 * q];
        acc[0][q] += z0 * w;
        acc[1][q] += z1 * w;
      }
    }
  }
  cp_async_wait<0>();
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    int col = c0 + tj + 32 * a;
    if (col >= d) continue;
    int64_t grow = pv.dofs[v] + col;
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
      int c = tc + 8 * q;
      if (c < NC) partG[((int64_t)blockIdx.x * D + grow) * NC + c] = acc64[a][q] + (double)acc[a][q];
    }
  }
}

__global__ void pass_reduce_kernel(const double* __restrict__ partG, int chunks, int64_t nG,
                                   const double* __restrict__ partGram, int ctas, int64_t nGram,
                                   double* __restrict__ G, double* __restrict__ Gram, const int* done) {
  if (done != nullptr && *done) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nG + nGram;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0;
    if (e < nG) {
      if (partG != nullptr) {
        for (int c = 0; c < chunks; ++c) s += (double)partG[(int64_t)c * nG + e];
        G[e] = s;
      }
    } else {
      int64_t f = e - nG;
      for (int c = 0; c < ctas; ++c) s += (double)partGram[(int64_t)c * nGram + f];
      Gram[f] = s;
    }
  }
}

// FDA: Xhat^T P = X^T P - sum_k m_k (sum_{i in k} P_i)^T.
__global__ void lda_correct_kernel(const double* __restrict__ partCls, int ctas, int l, int NC, int d,
                                   const double* __restrict__ means, double* __restrict__ G, const int* done) {
  __shared__ double sP[kMaxClasses * 48];
  if (done != nullptr && *done) return;
  for (int e = threadIdx.x; e < l * NC; e += blockDim.x) {
    double s = 0;
    for (int c = 0; c < ctas; ++c) s += (double)partCls[(int64_t)c * l * NC + e];
    sP[e] = s;
  }
  __syncthreads();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * NC; e += gridDim.x * blockDim.x) {
    int j = e / NC, c = e % NC;
    double corr = 0;
    for (int k = 0; k < l; ++k) corr += means[k * d + j] * sP[k * NC + c];
    G[e] -= corr;
  }
}

template <typename Tacc>
__global__ void phi_convert_kernel(const double* __restrict__ a, Tacc* __restrict__ b, int64_t len) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (Tacc)a[i];
}

// class-mean rows times Phi: Cls (l x NC) = means (l x d) Phi (d x 2k), FDA only
__global__ void lda_cls_kernel(const double* __restrict__ means, const double* __restrict__ Phi, int l,
                               int d, int k2, int stride, double* __restrict__ Cls) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= l * k2) return;
  int cls = e / k2, c = e % k2;
  double s = 0;
  for (int j = 0; j < d; ++j) s += means[(int64_t)cls * d + j] * Phi[(int64_t)j * stride + c];
  Cls[e] = s;
}

template <typename Tacc>
__global__ void cast_cls_kernel(const double* __restrict__ a, Tacc* __restrict__ b, int len) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) b[i] = (Tacc)a[i];
}

namespace {

template <typename Tin, typename Tacc, int RN>
int launch_w(Plan& p, const PassViews& pv, int NC, Tacc* W, cudaStream_t st, const Tacc* cls) {
  size_t smem = sizeof(Tacc) * (32 * (kTM + 1) + 32 * 8 * RN + kTM * NC) + sizeof(int) * kTM;
  auto kern = pass_w_kernel<Tin, Tacc, RN>;
  GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<p.ctasA, 256, smem, st>>>(pv, p.n, NC, W, reinterpret_cast<double*>(p.partGram),
                                    p.kind == kLDA ? p.labels : nullptr, cls, p.l,
                                    reinterpret_cast<double*>(p.partCls));
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

template <typename Tin, typename Tacc>
int dispatch_w(Plan& p, const PassViews& pv, int NC, Tacc* W, cudaStream_t st, const Tacc* cls) {
  int rn = (pv.k2 + 7) / 8;
  switch (rn) {
    case 1: return launch_w<Tin, Tacc, 1>(p, pv, NC, W, st, cls);
    case 2: return launch_w<Tin, Tacc, 2>(p, pv, NC, W, st, cls);
    case 3: return launch_w<Tin, Tacc, 3>(p, pv, NC, W, st, cls);
    case 4: return launch_w<Tin, Tacc, 4>(p, pv, NC, W, st, cls);
    default: return launch_w<Tin, Tacc, 5>(p, pv, NC, W, st, cls);
  }
}

template <typename Tin, typename Tacc, int RQ>
int launch_g(Plan& p, const PassViews& pv, const Tacc* W, cudaStream_t st) {
  int nb0 = ceil_div(pv.d[0], 64);
  int nb = nb0 + (pv.nviews > 1 ? ceil_div(pv.d[1], 64) : 0);
  int64_t rpc = (p.n + p.chunksB - 1) / p.chunksB;
  dim3 grid(p.chunksB, nb);
  pass_g_kernel<Tin, Tacc, RQ><<<grid, 256, 0, st>>>(pv, p.n, p.NC, p.D, W, rpc, nb0,
                                                      reinterpret_cast<double*>(p.partG));
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

template <int RQ>
int launch_g_async(Plan& p, const PassViews& pv, const float* W, cudaStream_t st) {
  int nb0 = ceil_div(pv.d[0], 64);
  int nb = nb0 + (pv.nviews > 1 ? ceil_div(pv.d[1], 64) : 0);
  int64_t rpc = (p.n + p.chunksB - 1) / p.chunksB;
  dim3 grid(p.chunksB, nb);
  const size_t smem = sizeof(float) * kGStages * kTB * (64 + 8 * RQ);
  auto kern = pass_g_async_kernel<RQ>;
  GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, 256, smem, st>>>(pv, p.n, p.NC, p.D, W, rpc, nb0, reinterpret_cast<double*>(p.partG));
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

// the pipelined FP32 kernel needs whole 16-byte chunks of every data row
bool g_async_eligible(const PassViews& pv) {
  for (int v = 0; v < pv.nviews; ++v)
    if (pv.d[v] % 4 != 0 || pv.ld[v] % 4 != 0 || (reinterpret_cast<uintptr_t>(pv.Z[v]) & 15) != 0) return false;
  return true;
}

template <typename Tin, typename Tacc>
int dispatch_g(Plan& p, const PassViews& pv, const Tacc* W, cudaStream_t st) {
  int rq = (p.NC + 7) / 8;
  if constexpr (std::is_same<Tin, float>::value && std::is_same<Tacc, float>::value) {
    if (g_async_eligible(pv)) {
      switch (rq) {
        case 1: return launch_g_async<1>(p, pv, W, st);
        case 2: return launch_g_async<2>(p, pv, W, st);
        case 3: return launch_g_async<3>(p, pv, W, st);
        case 4: return launch_g_async<4>(p, pv, W, st);
        case 5: return launch_g_async<5>(p, pv, W, st);
        case 6: return launch_g_async<6>(p, pv, W, st);
        case 7: return launch_g_async<7>(p, pv, W, st);
        case 8: return launch_g_async<8>(p, pv, W, st);
        case 9: return launch_g_async<9>(p, pv, W, st);
        default: return launch_g_async<10>(p, pv, W, st);
      }
    }
  }
  switch (rq) {
    case 1: return launch_g<Tin, Tacc, 1>(p, pv, W, st);
    case 2: return launch_g<Tin, Tacc, 2>(p, pv, W, st);
    case 3: return launch_g<Tin, Tacc, 3>(p, pv, W, st);
    case 4: return launch_g<Tin, Tacc, 4>(p, pv, W, st);
    case 5: return launch_g<Tin, Tacc, 5>(p, pv, W, st);
    case 6: return launch_g<Tin, Tacc, 6>(p, pv, W, st);
    case 7: return launch_g<Tin, Tacc, 7>(p, pv, W, st);
    case 8: return launch_g<Tin, Tacc, 8>(p, pv, W, st);
    case 9: return launch_g<Tin, Tacc, 9>(p, pv, W, st);
    default: return launch_g<Tin, Tacc, 10>(p, pv, W, st);
  }
}

template <typename Tin, typename Tacc>
int run_pass(Plan& p, bool gram_only, cudaStream_t st, int phi_cols, const int* done) {
  PassViews pv{};
  pv.nviews = p.nviews;
  pv.k2 = phi_cols;
  pv.phistride = 2 * p.k;
  pv.done = done;
  const int NC = p.nviews * phi_cols;
  int dofs = 0;
  for (int v = 0; v < p.nviews; ++v) {
    pv.Z[v] = p.v[v].Z;
    pv.ld[v] = p.v[v].ld;
    pv.d[v] = p.v[v].d;
    pv.dofs[v] = dofs;
    pv.ocol[v] = v * phi_cols;
    dofs += p.v[v].d;
    if (std::is_same<Tacc, double>::value) {
      pv.Phi[v] = p.v[v].Phi;
    } else {
      int64_t len = (int64_t)p.v[v].d * 2 * p.k;
      phi_convert_kernel<float><<<ceil_div(len, 256), 256, 0, st>>>(p.v[v].Phi, p.v[v].Phi32, len);
      GB_CHECK_LAUNCH();
      pv.Phi[v] = p.v[v].Phi32;
    }
  }
  Tacc* cls = nullptr;
  if (p.kind == kLDA) {
    int len = p.l * phi_cols;
    lda_cls_kernel<<<ceil_div(len, 128), 128, 0, st>>>(p.means, p.v[0].Phi, p.l, p.v[0].d, phi_cols, 2 * p.k,
                                                       p.Cls);
    GB_CHECK_LAUNCH();
    if (std::is_same<Tacc, double>::value) {
      cls = reinterpret_cast<Tacc*>(p.Cls);
    } else {
      cls = reinterpret_cast<Tacc*>(p.Cls + p.l * 2 * p.k);  // FP32 copy stored after the FP64 one
      cast_cls_kernel<Tacc><<<ceil_div(len, 128), 128, 0, st>>>(p.Cls, cls, len);
      GB_CHECK_LAUNCH();
    }
  }
  Tacc* W = gram_only ? nullptr : reinterpret_cast<Tacc*>(p.Wbuf);
  GB_TRY((dispatch_w<Tin, Tacc>(p, pv, NC, W, st, cls)));
  if (!gram_only) GB_TRY((dispatch_g<Tin, Tacc>(p, pv, W, st)));
  int64_t nG = gram_only ? 0 : (int64_t)p.D * NC;
  int64_t nGram = (int64_t)NC * NC;
  pass_reduce_kernel<<<ceil_div(nG + nGram, 256), 256, 0, st>>>(
      gram_only ? nullptr : reinterpret_cast<const double*>(p.partG), p.chunksB, nG,
      reinterpret_cast<const double*>(p.partGram), p.ctasA, nGram, p.G, p.Gram, done);
  GB_CHECK_LAUNCH();
  if (p.kind == kLDA && !gram_only) {
    lda_correct_kernel<<<ceil_div((int64_t)p.D * NC, 256), 256, 0, st>>>(
        reinterpret_cast<const double*>(p.partCls), p.ctasA, p.l, NC, p.D, p.means, p.G, done);
    GB_CHECK_LAUNCH();
  }
  return GBCCA_OK;
}

}  // namespace

// low = accumulate in FP32 (BF16/FP32 data); otherwise FP64.  gram_only
// skips Z^T W (the Rayleigh-Ritz refinement needs only W^T W).  phi_cols =
// columns of Phi used per view (0 = all 2k).  `done` (device, may be null)
// turns the launches into no-ops once the solver has stopped.
int fused_pass(Plan& p, bool low, bool gram_only, cudaStream_t st, int phi_cols, const int* done) {
  if (phi_cols <= 0) phi_cols = 2 * p.k;
  if (low && !gram_only && phi_cols == 2 * p.k && p.opt.tensor_cores) {
    if (p.tc_img != nullptr && tc_pass_eligible(p)) return tc_pass(p, st, done);
  }
  if (p.kev0 != nullptr) GB_CUDA(record_timing_event(p.kev0, st));
  const int rc = fused_pass_cores(p, low, gram_only, st, phi_cols, done);
  if (rc == GBCCA_OK && p.kev1 != nullptr) GB_CUDA(record_timing_event(p.kev1, st));
  return rc;
}

// CUDA-core passes (FP64 / FP32 data, LDA, and the BF16 plans the
// tensor-core pass does not serve)
int fused_pass_cores(Plan& p, bool low, bool gram_only, cudaStream_t st, int phi_cols, const int* done) {
  if (p.kind == kLDA && p.l * phi_cols > 256 * kCI) {
    set_last_error("too many classes x columns for the FDA pass");
    return GBCCA_ERR_UNSUPPORTED;
  }
  switch (p.dtype) {
    case GBCCA_FP64: return run_pass<double, double>(p, gram_only, st, phi_cols, done);
    case GBCCA_FP32:
      return low ? run_pass<float, float>(p, gram_only, st, phi_cols, done)
                 : run_pass<float, double>(p, gram_only, st, phi_cols, done);
    case GBCCA_BF16:
      return low ? run_pass<__nv_bfloat16, float>(p, gram_only, st, phi_cols, done)
                 : run_pass<__nv_bfloat16, double>(p, gram_only, st, phi_cols, done);
  }
  return GBCCA_ERR_INVALID_ARG;
}

// ------------------------------------------------------------ FDA statistics
// Per-class column sums in FP64: CTA = (row chunk, 256-column block); each
// thread owns one column, so the accumulation order is fixed.
template <typename Tin>
__global__ void class_sums_kernel(const Tin* __restrict__ X, int64_t ld, int64_t n, int d,
                                  const int32_t* __restrict__ y, int l, int64_t rows_per_chunk,
                                  double* __restrict__ part, double* __restrict__ cnt_part) {
  extern __shared__ double acc[];  // [l][256]
  const int c = blockIdx.y * 256 + threadIdx.x;
  for (int k = 0; k < l; ++k) acc[k * 256 + threadIdx.x] = 0;
  const int64_t r0 = blockIdx.x * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
  if (c < d)
    for (int64_t i = r0; i < r1; ++i) {
      const int yi = y[i];
      if (yi >= 0 && yi < l) acc[yi * 256 + threadIdx.x] += to_f64(X[i * ld + c]);  // bad labels: see label_check
    }
  if (c < d)
    for (int k = 0; k < l; ++k) part[((int64_t)blockIdx.x * l + k) * d + c] = acc[k * 256 + threadIdx.x];
  if (blockIdx.y == 0 && threadIdx.x < l) {
    double cn = 0;
    for (int64_t i = r0; i < r1; ++i) cn += (y[i] == (int)threadIdx.x) ? 1.0 : 0.0;
    cnt_part[(int64_t)blockIdx.x * l + threadIdx.x] = cn;
  }
}

__global__ void class_finish_kernel(const double* __restrict__ part, const double* __restrict__ cnt_part,
                                    int chunks, int l, int d, double* __restrict__ counts,
                                    double* __restrict__ means, double* __restrict__ Yhat, int* flag) {
  __shared__ double cn[kMaxClasses];
  if (threadIdx.x < l) {
    double s = 0;
    for (int c = 0; c < chunks; ++c) s += cnt_part[(int64_t)c * l + threadIdx.x];
    cn[threadIdx.x] = s;
    if (blockIdx.x == 0) {
      counts[threadIdx.x] = s;
      if (s <= 0) atomicExch(flag, kFlagNotSpd);
    }
  }
  __syncthreads();
  double ntot = 0;
  for (int k = 0; k < l; ++k) ntot += cn[k];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x) {
    double tot = 0;
    for (int k = 0; k < l; ++k) {
      double s = 0;
      for (int c = 0; c < chunks; ++c) s += part[((int64_t)c * l + k) * d + j];
      means[k * d + j] = cn[k] > 0 ? s / cn[k] : 0.0;
      tot += s;
    }
    double m = tot / ntot;
    for (int k = 0; k < l; ++k) Yhat[k * d + j] = sqrt(cn[k]) * (means[k * d + j] - m);
  }
}

// Every label in [0, l): the later kernels index class tables by label.
__global__ void label_check_kernel(const int32_t* __restrict__ y, int64_t n, int l, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (y[i] < 0 || y[i] >= l) atomicExch(flag, kFlagLabel);
}

int lda_class_stats(Plan& p, cudaStream_t st) {
  label_check_kernel<<<std::min(ceil_div(p.n, 256), 4 * p.sm_count), 256, 0, st>>>(p.labels, p.n, p.l, p.flag);
  GB_CHECK_LAUNCH();
  const int chunks = 128;
  int64_t rpc = (p.n + chunks - 1) / chunks;
  dim3 grid(chunks, ceil_div(p.D, 256));
  size_t smem = sizeof(double) * p.l * 256;
  double* part = p.clsPart;
  double* cnt = p.clsPart + (int64_t)chunks * p.l * p.D;
  switch (p.dtype) {
    case GBCCA_FP64: {
      auto kern = class_sums_kernel<double>;
      GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<grid, 256, smem, st>>>((const double*)p.v[0].Z, p.v[0].ld, p.n, p.D, p.labels, p.l, rpc, part, cnt);
      break;
    }
    case GBCCA_FP32: {
      auto kern = class_sums_kernel<float>;
      GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<grid, 256, smem, st>>>((const float*)p.v[0].Z, p.v[0].ld, p.n, p.D, p.labels, p.l, rpc, part, cnt);
      break;
    }
    default: {
      auto kern = class_sums_kernel<__nv_bfloat16>;
      GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<grid, 256, smem, st>>>((const __nv_bfloat16*)p.v[0].Z, p.v[0].ld, p.n, p.D, p.labels, p.l, rpc,
                                    part, cnt);
    }
  }
  GB_CHECK_LAUNCH();
  class_finish_kernel<<<ceil_div(p.D, 256), 256, 0, st>>>(part, cnt, chunks, p.l, p.D, p.counts, p.means,
                                                          p.Yhat, p.flag);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

}  // namespace gbcca
