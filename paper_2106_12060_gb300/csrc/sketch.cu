// Sketching transforms S Z for the preconditioner (Sec. 3, App. A).
//
// CountSketch (Sec. 3): row i of Z, times g(i) = +-1, is added into row h(i)
// of S Z.  The rows are first grouped by bucket with a stable counting sort
// (per-chunk counters, a bucket-major prefix sum, then an in-order placement
// with warp match), and each bucket is summed by one warp in row order in
// FP64, so the sketch is bitwise reproducible.
//
// SRHT (App. A, Def. A.1, scale sqrt(n/s) so that E[S^T S] = I): the
// Walsh-Hadamard transform of length n_pad = 2^m factors as
// H_{2^m} = H_{N2} (x) H_{N1}; stage 1 transforms each block of N1 consecutive
// rows in shared memory, stage 2 transforms the strided columns of the
// intermediate and writes only the s sampled rows.
#include "plan.h"

namespace gbcca {

// --------------------------------------------------------------- draws
__device__ __forceinline__ uint64_t feistel_even(uint64_t x, int bits, uint64_t key) {
  const int half = bits / 2;
  const uint64_t mask = (1ull << half) - 1ull;
  uint64_t L = (x >> half) & mask, R = x & mask;
  for (int r = 0; r < 4; ++r) {
    uint64_t F = sm64(key, (uint64_t)r ^ (R << 8)) & mask;
    uint64_t nL = R, nR = L ^ F;
    L = nL;
    R = nR;
  }
  return (L << half) | R;
}

__global__ void draw_countsketch_kernel(int64_t n, int64_t s, uint64_t seed, int32_t* h, int8_t* g) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t r = sm64(seed, (uint64_t)i);
    h[i] = (int32_t)(((r >> 32) * (uint64_t)s) >> 32);
    g[i] = (r & 1ull) ? (int8_t)-1 : (int8_t)1;
  }
}

__global__ void draw_srht_kernel(int64_t n_pad, int m, int64_t s, uint64_t seed, int32_t* rows, int8_t* signs,
                                 int* flag) {
  const uint64_t kd = seed ^ kSaltSigns, kr = seed ^ kSaltRows;
  const int bits = (m % 2 == 0) ? m : m + 1;
  const uint64_t lim = 1ull << m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * blockDim.x) {
    signs[i] = (sm64(kd, (uint64_t)i) & 1ull) ? (int8_t)-1 : (int8_t)1;
    if (i < s) {
      uint64_t y = feistel_even((uint64_t)i, bits, kr);
      // cycle walking: the orbit of i under the permutation returns to i < 2^m,
      // so the loop ends; the bound only guards against a broken build.
      int guard = 0;
      while (y >= lim && guard < (1 << 22)) {
        y = feistel_even(y, bits, kr);
        ++guard;
      }
      if (y >= lim && flag != nullptr) atomicExch(flag, kFlagDraw);
      rows[i] = (int32_t)y;
    }
  }
}

int sketch_draws(int kind, int64_t n, int64_t s, uint64_t seed, int32_t* h, int8_t* g, cudaStream_t st) {
  if (kind == GBCCA_SKETCH_COUNTSKETCH) {
    draw_countsketch_kernel<<<std::min(ceil_div(n, 256), 8192), 256, 0, st>>>(n, s, seed, h, g);
    GB_CHECK_LAUNCH();
    return GBCCA_OK;
  }
  if (kind == GBCCA_SKETCH_SRHT) {
    int m = 0;
    while ((1ll << m) < n) ++m;
    if ((1ll << m) != n || s > n) {
      set_last_error("SRHT draws need n a power of two and s <= n");
      return GBCCA_ERR_INVALID_ARG;
    }
    draw_srht_kernel<<<std::min(ceil_div(n, 256), 8192), 256, 0, st>>>(n, m, s, seed, h, g, nullptr);
    GB_CHECK_LAUNCH();
    return GBCCA_OK;
  }
  set_last_error("unknown sketch kind");
  return GBCCA_ERR_INVALID_ARG;
}

// ---------------------------------------------------- CountSketch sort
__global__ void cs_count_kernel(const int32_t* __restrict__ h, int64_t n, int64_t rpc, int64_t s,
                                int32_t* __restrict__ tab, int* flag) {
  const int64_t r0 = blockIdx.x * rpc, r1 = min(n, r0 + rpc);
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    int32_t b = h[i];
    if (b < 0 || b >= s) {
      atomicExch(flag, kFlagBucket);
      continue;
    }
    atomicAdd(&tab[(int64_t)blockIdx.x * s + b], 1);
  }
}

// per bucket: exclusive prefix over chunks (in place) and the bucket total
__global__ void cs_colscan_kernel(int32_t* __restrict__ tab, int nch, int64_t s, int32_t* __restrict__ total) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < s; b += (int64_t)gridDim.x * blockDim.x) {
    int32_t acc = 0;
    for (int c = 0; c < nch; ++c) {
      int32_t t = tab[(int64_t)c * s + b];
      tab[(int64_t)c * s + b] = acc;
      acc += t;
    }
    total[b] = acc;
  }
}

// exclusive scan of total[0..s) into off[0..s] by one CTA of 1024 threads
__global__ void cs_scan_kernel(const int32_t* __restrict__ total, int64_t s, int32_t* __restrict__ off) {
  __shared__ int32_t buf[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < s; base += 1024) {
    int64_t i = base + threadIdx.x;
    int32_t v = i < s ? total[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int32_t t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < s) off[i] = carry + buf[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) off[s] = carry;
}

// in-order placement: one warp walks its chunk 32 rows at a time; rows of
// the same bucket inside a group of 32 are ranked by lane (= row) order.
__global__ void cs_place_kernel(const int32_t* __restrict__ h, int64_t n, int64_t rpc, int64_t s,
                                int32_t* __restrict__ tab, const int32_t* __restrict__ off,
                                int32_t* __restrict__ perm) {
  const int lane = threadIdx.x;
  const int64_t r0 = blockIdx.x * rpc, r1 = min(n, r0 + rpc);
  int32_t* cur = tab + (int64_t)blockIdx.x * s;
  for (int64_t i0 = r0; i0 < r1; i0 += 32) {
    const int64_t i = i0 + lane;
    int32_t b = -1;
    if (i < r1) {
      b = h[i];
      if (b < 0 || b >= s) b = -1;  // reported by cs_count_kernel
    }
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const bool act = b >= 0;
    const bool last = act && (peers >> lane) == 1u;  // highest lane of its group
    if (act) {
      const int rank = __popc(peers & ((1u << lane) - 1u));
      perm[off[b] + cur[b] + rank] = (int32_t)i;
    }
    __syncwarp();
    if (last) cur[b] += __popc(peers);
    __syncwarp();
  }
}

int countsketch_prepare(Plan& p, cudaStream_t st) {
  const int64_t rpc = (p.n + p.cs_nch - 1) / p.cs_nch;
  GB_CUDA(cudaMemsetAsync(p.cs_tab, 0, sizeof(int32_t) * (size_t)p.cs_nch * p.s, st));
  cs_count_kernel<<<p.cs_nch, 256, 0, st>>>(p.h, p.n, rpc, p.s, p.cs_tab, p.flag);
  GB_CHECK_LAUNCH();
  int32_t* total = p.perm;  // borrow perm as scratch for the bucket totals (n >= s)
  cs_colscan_kernel<<<ceil_div(p.s, 256), 256, 0, st>>>(p.cs_tab, p.cs_nch, p.s, total);
  GB_CHECK_LAUNCH();
  cs_scan_kernel<<<1, 1024, 0, st>>>(total, p.s, p.cs_off);
  GB_CHECK_LAUNCH();
  cs_place_kernel<<<p.cs_nch, 32, 0, st>>>(p.h, p.n, rpc, p.s, p.cs_tab, p.cs_off, p.perm);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

// one warp per bucket; each lane owns columns lane, lane + 32, ...
template <typename Tin>
__global__ void __launch_bounds__(256)
cs_sum_kernel(const Tin* __restrict__ Z, int64_t ld, int d, int64_t s, const int32_t* __restrict__ off,
              const int32_t* __restrict__ perm, const int8_t* __restrict__ g, const int32_t* __restrict__ labels,
              const double* __restrict__ means, double* __restrict__ SZ) {
  const int lane = threadIdx.x & 31;
  const int64_t b = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (b >= s) return;
  double acc[kMaxD / 32];
#pragma unroll
  for (int q = 0; q < kMaxD / 32; ++q) acc[q] = 0.0;
  const int nq = (d + 31) / 32;
  for (int32_t pos = off[b]; pos < off[b + 1]; ++pos) {
    const int32_t i = perm[pos];
    const double sg = (double)g[i];
    const Tin* row = Z + (int64_t)i * ld;
    const double* mrow = labels != nullptr ? means + (int64_t)labels[i] * d : nullptr;
#pragma unroll
    for (int q = 0; q < kMaxD / 32; ++q) {
      int c = lane + 32 * q;
      if (q < nq && c < d) {
        double x = to_f64(row[c]);
        if (mrow != nullptr) x -= mrow[c];
        acc[q] += sg * x;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kMaxD / 32; ++q) {
    int c = lane + 32 * q;
    if (q < nq && c < d) SZ[b * d + c] = acc[q];
  }
}

int countsketch_apply(Plan& p, int view, bool center, cudaStream_t st) {
  View& v = p.v[view];
  const int32_t* lab = center ? p.labels : nullptr;
  const double* mean = center ? p.means : nullptr;
  int grid = ceil_div(p.s, 8);
  switch (p.dtype) {
    case GBCCA_FP64:
      cs_sum_kernel<double><<<grid, 256, 0, st>>>((const double*)v.Z, v.ld, v.d, p.s, p.cs_off, p.perm, p.g, lab,
                                                  mean, v.SZ);
      break;
    case GBCCA_FP32:
      cs_sum_kernel<float><<<grid, 256, 0, st>>>((const float*)v.Z, v.ld, v.d, p.s, p.cs_off, p.perm, p.g, lab, mean,
                                                 v.SZ);
      break;
    default:
      cs_sum_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16*)v.Z, v.ld, v.d, p.s, p.cs_off, p.perm,
                                                         p.g, lab, mean, v.SZ);
  }
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

// ---------------------------------------------------------------- SRHT
constexpr int kLoadBatch = 8;

// Unnormalized Walsh-Hadamard transform of one column of length N (32 <= N
// <= 1024, power of two) held in shared memory with row stride `stride`, by
// one warp: lane l holds rows l + 32 t; butterflies of span < 32 go across
// lanes (shuffles), larger spans within the lane's registers.
template <typename T, int NT>
__device__ __forceinline__ void fwht_warp_col_n(T* col, int stride) {
  const int lane = threadIdx.x & 31;
  T v[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) v[t] = col[(lane + 32 * t) * stride];
#pragma unroll
  for (int h = 1; h < 32; h <<= 1) {
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const T x = v[t];
      const T y = __shfl_xor_sync(0xffffffffu, x, h);
      v[t] = (lane & h) ? (y - x) : (x + y);
    }
  }
#pragma unroll
  for (int hb = 1; hb < NT; hb <<= 1) {  // span 32 hb rows = hb register slots
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      if ((t & hb) == 0) {
        const T a = v[t], b = v[t + hb];
        v[t] = a + b;
        v[t + hb] = a - b;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) col[(lane + 32 * t) * stride] = v[t];
}

template <typename T>
__device__ __forceinline__ void fwht_warp_col(T* col, int stride, int N) {
  switch (N >> 5) {
    case 1: fwht_warp_col_n<T, 1>(col, stride); break;
    case 2: fwht_warp_col_n<T, 2>(col, stride); break;
    case 4: fwht_warp_col_n<T, 4>(col, stride); break;
    case 8: fwht_warp_col_n<T, 8>(col, stride); break;
    case 16: fwht_warp_col_n<T, 16>(col, stride); break;
    default: fwht_warp_col_n<T, 32>(col, stride); break;
  }
}

// Transform of length N < 32 (tiny n): one thread per column
template <typename T>
__device__ __forceinline__ void fwht_thread_col(T* col, int stride, int N) {
  for (int h = 1; h < N; h <<= 1)
    for (int i = 0; i < N; ++i)
      if ((i & h) == 0) {
        const T a = col[i * stride], b = col[(i + h) * stride];
        col[i * stride] = a + b;
        col[(i + h) * stride] = a - b;
      }
}

// Stage 1: per block of N1 consecutive rows and CB = 32 columns, D Z
// (signs, and the class means for LDA) then the N1-point transform along the
// rows of each column, written to the intermediate buffer.  Tile in shared
// memory as [N1][33] (padded: column reads are conflict-free); FP32 data is
// converted on FP32 units.
template <typename Tin, typename T>
__global__ void __launch_bounds__(512)
srht_stage1_kernel(const Tin* __restrict__ Z, int64_t ld, int64_t n, int d, int N1, const int8_t* __restrict__ sg,
                   const int32_t* __restrict__ labels, const double* __restrict__ means, T* __restrict__ Tmid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* buf = reinterpret_cast<T*>(smem_raw);
  constexpr int CB = 32, LD = 33;
  const int64_t i2 = blockIdx.y;   // column blocks of one row block run next to each other
  const int c0 = blockIdx.x * CB;
  // loads batched (kLoadBatch in flight per thread), then signs and stores
  for (int base = 0; base < N1 * CB; base += blockDim.x * kLoadBatch) {
    Tin z[kLoadBatch];
    int8_t g[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int e = base + threadIdx.x + blockDim.x * u;
      const int r = e >> 5, c = e & 31;
      const int64_t row = i2 * N1 + r;
      const bool in = e < N1 * CB && row < n && c0 + c < d;
      z[u] = in ? Z[row * ld + c0 + c] : Tin(0.0f);
      g[u] = in ? sg[row] : int8_t(0);
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int e = base + threadIdx.x + blockDim.x * u;
      if (e >= N1 * CB) continue;
      const int r = e >> 5, c = e & 31;
      const int64_t row = i2 * N1 + r;
      T val = T(0);
      if (g[u] != 0) {
        if (labels != nullptr) {
          const double x = to_f64(z[u]) - means[(int64_t)labels[row] * d + c0 + c];
          val = (T)(g[u] < 0 ? -x : x);
        } else {
          const T x = to_work<T>(z[u]);
          val = g[u] < 0 ? -x : x;
        }
      }
      buf[r * LD + c] = val;
    }
  }
  __syncthreads();
  if (N1 >= 32) {
    for (int c = threadIdx.x >> 5; c < CB; c += blockDim.x >> 5) fwht_warp_col<T>(buf + c, LD, N1);
  } else if (threadIdx.x < CB) {
    fwht_thread_col<T>(buf + threadIdx.x, LD, N1);
  }
  __syncthreads();
  // intermediate row r * N2 + i2: stage 2 then reads N2 consecutive rows
  const int64_t N2 = gridDim.y;
  for (int e = threadIdx.x; e < N1 * CB; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    if (c0 + c < d) Tmid[((int64_t)r * N2 + i2) * d + c0 + c] = buf[r * LD + c];
  }
}

// Stage 2: for one residue a1 of the low m1 row bits, the N2-point transform
// across the row blocks of each column, kept only at the sampled rows and
// scaled by sqrt(n'/s) / sqrt(n') = 1 / sqrt(s) (App. A).
template <typename T>
__global__ void __launch_bounds__(512)
srht_stage2_kernel(const T* __restrict__ Tmid, int d, int N1, int N2, int m1, const int32_t* __restrict__ off1,
                   const int32_t* __restrict__ list, const int32_t* __restrict__ rows, double scale,
                   double* __restrict__ SZ) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* buf = reinterpret_cast<T*>(smem_raw);
  constexpr int CB = 32, LD = 33;
  const int a1 = blockIdx.y;
  const int c0 = blockIdx.x * CB;
  const int nsel = off1[a1 + 1] - off1[a1];
  if (nsel == 0) return;
  for (int base = 0; base < N2 * CB; base += blockDim.x * kLoadBatch) {
    T v[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int e = base + threadIdx.x + blockDim.x * u;
      const int r = e >> 5, c = e & 31;
      v[u] = (e < N2 * CB && c0 + c < d) ? Tmid[((int64_t)a1 * N2 + r) * d + c0 + c] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int e = base + threadIdx.x + blockDim.x * u;
      if (e < N2 * CB) buf[(e >> 5) * LD + (e & 31)] = v[u];
    }
  }
  __syncthreads();
  if (N2 >= 32) {
    for (int c = threadIdx.x >> 5; c < CB; c += blockDim.x >> 5) fwht_warp_col<T>(buf + c, LD, N2);
  } else if (threadIdx.x < CB) {
    fwht_thread_col<T>(buf + threadIdx.x, LD, N2);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nsel * CB; e += blockDim.x) {
    const int q = e >> 5, c = e & 31;
    const int j = list[off1[a1] + q];
    const int a2 = rows[j] >> m1;
    if (c0 + c < d) SZ[(int64_t)j * d + c0 + c] = scale * (double)buf[a2 * LD + c];
  }
}

// group the sampled rows by their low m1 bits (order within a group is free:
// every sampled row writes its own output row)
__global__ void srht_group_kernel(const int32_t* __restrict__ rows, int64_t s, int N1, int32_t* __restrict__ cnt,
                                  int32_t* __restrict__ off1, int32_t* __restrict__ list, int phase) {
  if (phase == 0) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < s; j += (int64_t)gridDim.x * blockDim.x)
      atomicAdd(&cnt[rows[j] & (N1 - 1)], 1);
  } else if (phase == 1) {
    // exclusive scan of the N1 counts by one warp: lane l sums a contiguous
    // run of the counts, the lanes' totals are scanned by shuffles, then
    // each lane writes its run's offsets (and clears its counts)
    if (blockIdx.x == 0 && threadIdx.x < 32) {
      const int lane = threadIdx.x;
      const int per = (N1 + 31) / 32;
      const int a0 = min(N1, lane * per), a1 = min(N1, a0 + per);
      int32_t tot = 0;
      for (int a = a0; a < a1; ++a) tot += cnt[a];
      int32_t inc = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      int32_t acc = inc - tot;
      for (int a = a0; a < a1; ++a) {
        off1[a] = acc;
        acc += cnt[a];
        cnt[a] = 0;
      }
      if (lane == 31) off1[N1] = inc;
    }
  } else {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < s; j += (int64_t)gridDim.x * blockDim.x) {
      int a = rows[j] & (N1 - 1);
      int pos = atomicAdd(&cnt[a], 1);
      list[off1[a] + pos] = (int32_t)j;
    }
  }
}

template <typename Tin, typename T>
int srht_run(Plan& p, View& v, cudaStream_t st) {
  constexpr int CB = 32;
  int m = 0;
  while ((1ll << m) < p.n_pad) ++m;
  const int m1 = std::min(m, 9), m2 = m - m1;
  const int N1 = 1 << m1, N2 = 1 << m2;
  if (N2 > 1024) {
    set_last_error("SRHT supports n <= 2^19");
    return GBCCA_ERR_UNSUPPORTED;
  }
  T* Tmid = reinterpret_cast<T*>(p.srht_T);
  const int32_t* lab = p.kind == kLDA ? p.labels : nullptr;
  size_t sm1 = sizeof(T) * N1 * (CB + 1);
  auto k1 = srht_stage1_kernel<Tin, T>;
  GB_CUDA(cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
  k1<<<dim3(ceil_div(v.d, CB), N2), 512, sm1, st>>>((const Tin*)v.Z, v.ld, p.n, v.d, N1, p.g, lab, p.means, Tmid);
  GB_CHECK_LAUNCH();
  int32_t* cnt = p.cs_tab;
  int32_t* off1 = p.cs_off;
  int32_t* list = p.perm;
  GB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * N1, st));
  srht_group_kernel<<<ceil_div(p.s, 256), 256, 0, st>>>(p.h, p.s, N1, cnt, off1, list, 0);
  GB_CHECK_LAUNCH();
  srht_group_kernel<<<1, 32, 0, st>>>(p.h, p.s, N1, cnt, off1, list, 1);
  GB_CHECK_LAUNCH();
  srht_group_kernel<<<ceil_div(p.s, 256), 256, 0, st>>>(p.h, p.s, N1, cnt, off1, list, 2);
  GB_CHECK_LAUNCH();
  size_t sm2 = sizeof(T) * N2 * (CB + 1);
  auto k2 = srht_stage2_kernel<T>;
  GB_CUDA(cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
  k2<<<dim3(ceil_div(v.d, CB), N1), 512, sm2, st>>>(Tmid, v.d, N1, N2, m1, off1, list, p.h,
                                                     1.0 / sqrt((double)p.s), v.SZ);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

int srht_apply(Plan& p, int view, cudaStream_t st) {
  View& v = p.v[view];
  switch (p.dtype) {
    case GBCCA_FP64: return srht_run<double, double>(p, v, st);
    case GBCCA_FP32: return srht_run<float, float>(p, v, st);
    default: return srht_run<__nv_bfloat16, float>(p, v, st);
  }
}

}  // namespace gbcca
