// BF16 hi/lo copy of FP32 data for the tensor-core pass (Sec. 4.2 gradient
// and Sec. 5.1-5.2 for the products the pass forms; Cor. 4.6 and Cor. 5.6
// for their one read of the data per iteration).
//
// When FP32 data is bound to a plan, each view Z is stored once more as a
// row-interleaved BF16 matrix of 2n rows: row 2i = bf16(z_i), row 2i + 1 =
// bf16(z_i - bf16(z_i)).  The two rows of a data row sum to it within 2^-17
// relative per element (z in [2^e, 2^(e+1)): |z - hi| <= 2^(e-8), and
// rounding the remainder to 8 bits errs by at most 2^(e-17)), and they take
// the 4 bytes per element of the FP32 data.  For FDA the copy is made of the
// class-centred rows Xhat = X - M[y] (Sec. 5.1), so that the pass needs no
// class-mean correction: S_w Phi = Xhat^T (Xhat Phi).  Products of BF16
// operands are exact in FP32, so the pass (pass_tc.cu) computes the products
// of this fixed representation with FP32 accumulation; its epilogue adds the
// two product rows of each data row.
#include <cuda_bf16.h>

#include "common.cuh"
#include "plan.h"

namespace gbcca {

namespace {

// Row i of the data (FDA: minus its class mean) goes to rows 2i (hi) and
// 2i + 1 (lo) of the copy, leading dimension ldo.
__global__ void hilo_copy_kernel(const float* __restrict__ Z, int64_t ld, int64_t n, int d,
                                 const int32_t* __restrict__ y, const double* __restrict__ means,
                                 __nv_bfloat16* __restrict__ out, int64_t ldo) {
  const int64_t total = n * (int64_t)d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / d;
    const int j = (int)(e - i * d);
    double v = (double)Z[i * ld + j];
    if (y != nullptr) v -= means[(int64_t)y[i] * d + j];
    const __nv_bfloat16 h = __double2bfloat16(v);
    out[2 * i * ldo + j] = h;
    out[(2 * i + 1) * ldo + j] = __double2bfloat16(v - (double)__bfloat162float(h));
  }
}

// Shapes the tensor-core pass streams through the copy: FP32 CCA of any
// shape the library accepts (d <= 1024, k <= 20); FP32 FDA with d <= 1024
bool hilo_shape_ok(const Plan& p) {
  if (p.dtype != GBCCA_FP32) return false;
  return p.kind == kCCA || p.v[0].d <= 1024;
}

}  // namespace

int hilo_alloc(Plan& p) {
  p.ts_ready = false;
  if (!p.opt.tensor_cores || !hilo_shape_ok(p)) return GBCCA_OK;
  for (int v = 0; v < p.nviews; ++v) {
    // rows padded to 16 bytes (the TMA row stride)
    const int64_t ldo = (p.v[v].d + 7) / 8 * 8;
    p.ts_ld[v] = ldo;
    void* t = nullptr;
    if (counted_malloc(&t, sizeof(__nv_bfloat16) * (size_t)2 * p.n * ldo) != cudaSuccess) {
      cudaGetLastError();
      set_last_error("allocation of the BF16 hi/lo copy of the data failed");
      return GBCCA_ERR_OOM;
    }
    p.ts_copy[v] = static_cast<__nv_bfloat16*>(t);
  }
  return GBCCA_OK;
}

// Makes the copies of the bound data (FDA: of the class-centred rows, after
// the class statistics).
int hilo_prepare(Plan& p, cudaStream_t st) {
  p.ts_ready = false;
  if (!p.opt.tensor_cores || p.ts_copy[0] == nullptr) return GBCCA_OK;
  for (int v = 0; v < p.nviews; ++v) {
    const int d = p.v[v].d;
    const int64_t total = p.n * (int64_t)d;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 8 * (int64_t)p.sm_count);
    hilo_copy_kernel<<<grid, 256, 0, st>>>(static_cast<const float*>(p.v[v].Z), p.v[v].ld, p.n, d,
                                           p.kind == kLDA ? p.labels : nullptr, p.kind == kLDA ? p.means : nullptr,
                                           p.ts_copy[v], p.ts_ld[v]);
    GB_CHECK_LAUNCH();
  }
  p.ts_ready = true;
  return GBCCA_OK;
}

}  // namespace gbcca
