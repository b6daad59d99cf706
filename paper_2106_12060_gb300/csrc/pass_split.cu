// Tensor-core (tcgen05 + TMA) fused data pass for FP32 data on sm_103a: the
// CCA pass (Sec. 4.2 gradient, Cor. 4.6 cost O(p (nnz X + nnz Y)) per
// iteration) and the FDA pass (Sec. 5.1-5.2, Cor. 5.6), both reading the data
// once per iteration.
//
// Representation.  When the data is bound to the plan, each FP32 view Z is
// stored once more as two BF16 matrices Z_hi = bf16(Z), Z_lo = bf16(Z - Z_hi)
// (together 4 bytes per element, the bytes of the FP32 data; Z_hi + Z_lo
// equals Z to 2^-17 relative per element).  For FDA the copy is made of the
// class-centred rows Xhat = X - M[y] (Sec. 5.1), so that the pass needs no
// class-mean correction: S_w Phi = Xhat^T (Xhat Phi).  Products of BF16
// operands are exact in FP32, so the pass is the products of this fixed
// representation with FP32 accumulation.
//
// Each 2-CTA cluster takes 32-row tiles.  CCA: CTA v streams view v as the
// two parts [Z_hi | Z_lo]; FDA: CTA 0 streams Xhat_hi, CTA 1 Xhat_lo.  Per
// tile and CTA:
//   GEMM 1  P = part tiles x Phi_v (tcgen05, M = 64 of which rows 0..31 are
//           the tile, N = 2h: Phi as bf16 hi | lo columns), two issuers into
//           two TMEM accumulators;
//   exchange the epilogue's data threads (one tile row each) add hi/lo
//           columns and accumulators, keep their P row in registers and store
//           it into the peer CTA's exchange buffer (st.shared::cluster, then
//           a release arrive on the peer's barrier); after the peer's row
//           has arrived they form W (CCA: [P_x | P_y]; FDA: P_0 + P_1 in
//           rank order, identical in both CTAs), split it into bf16 hi + lo
//           and write the K-major B operand of GEMM 2 in their own CTA;
//   GEMM 2  G_v += part tiles^T [W_hi | W_lo] (M = 128 columns of the part,
//           read MN-major from the same shared-memory boxes, N = 2 NW,
//           K = 32 rows), the hi and lo parts of the data accumulating into
//           the same TMEM accumulator.
// At the end the epilogue drains G to per-cluster (CCA) or per-CTA (FDA)
// FP32 partials; tc_reduce_kernel sums them in fixed order.
//
// Every remote operation is synchronous (DSMEM stores and remote mbarrier
// arrives, ordered by release/acquire at cluster scope); the only
// asynchronous operations are each CTA's own TMA loads and MMAs.  Every wait
// is bounded (a plan option sets the bound); a CTA whose wait runs out sets an
// abort flag that ends all its roles, drains its own TMA loads and MMAs
// (bounded), zeroes its partial, records the error code and meets its peer
// at a final cluster barrier, after which no operation targets either CTA.
#include "tc_ptx.cuh"

namespace gbcca {

namespace ts {
using namespace tc;

constexpr int kRows = 32;            // rows per tile (valid rows of GEMM 1's M = 64; K of GEMM 2)
constexpr int kBox = 4096;           // one 32-row x 64-column BF16 box
constexpr int kSlot = 2 * kBox;      // a pair of boxes: 128 columns of a tile
constexpr int kH = 20;               // W rows per view in the operands (2k <= 20)
constexpr int kN1 = 2 * kH;          // N of GEMM 1: Phi hi | lo
constexpr int kKBox1 = kN1 * 128;    // one K-box (64 columns) of the Phi image
constexpr int kTW = 48;              // TMEM column stride of the GEMM 1 accumulators
constexpr int kD1Cols = 48;          // TMEM columns read back for P
constexpr int kXC = 20;              // floats per row in the exchange buffer
constexpr int kMaxSmem = 232448;
constexpr uint32_t kTmemCols = 512;
constexpr int kPhiStride = 16 * kKBox1;  // per-view stride of the Phi images in the plan buffer

// GEMM 2's B operand holds the hi rows of W, then its lo rows.  CCA (W has
// 2 x 2k <= 40 columns): one MMA with N = 80 covers both parts, whose
// products accumulate in separate TMEM columns added at the drain.  FDA (W
// has 2k <= 20 columns, rows padded to 32): two MMAs with N = 32 per K step,
// hi then lo, into the same accumulator (an MMA with M = 128 needs N a
// multiple of 16, and TMEM holds 7 such accumulators of 32 columns).
template <bool kLda>
struct SLay {
  static constexpr int kMaxPairs = kLda ? 7 : 4;           // 128-column pairs of one part
  static constexpr int kParts = kLda ? 1 : 2;              // parts a CTA streams
  static constexpr int kPhiBytes = 2 * kMaxPairs * kKBox1;
  static constexpr int kNW = kLda ? 32 : 2 * kH;           // rows of one part (hi or lo) of W's operand
  static constexpr int kN2 = kLda ? kNW : 2 * kNW;         // N of one GEMM 2 MMA = TMEM columns of a G accumulator
  static constexpr int kWs = kNW * 128;
  static constexpr int kWBuf = 2 * kWs;
  static constexpr int kXBuf = kRows * kXC * 4;            // the peer's P rows of one tile
  static constexpr int kTG = 4 * kTW;                      // first TMEM column of the G accumulators
  static constexpr int kStages = (kMaxSmem - kPhiBytes - 2 * kWBuf - 2 * kXBuf - 512 - 1024) / kSlot;
  // the ring comes first: GEMM 1 reads 64 rows (4 KB past a box), which must
  // stay inside this CTA's shared memory
  static constexpr int kPhiOff = kStages * kSlot;
  static constexpr int kWsOff = kPhiOff + kPhiBytes;
  static constexpr int kXOff = kWsOff + 2 * kWBuf;
  static constexpr int kBarOff = kXOff + 2 * kXBuf;
  static constexpr int kSmemBytes = kBarOff + 512 + 1024;
  static constexpr int kFull = 0, kEmpty = kStages, kD1Full = 2 * kStages, kD1Free = kD1Full + 2;
  static constexpr int kXFull = kD1Free + 2, kXFree = kXFull + 2, kWReady = kXFree + 2, kWFree = kWReady + 2;
  static constexpr int kGDone = kWFree + 2, kFinal = kGDone + 1, kPhiFull = kFinal + 3;
  static constexpr int kNumBars = kPhiFull + 1;
  static_assert(kStages >= 2 * kParts * kMaxPairs, "two resident tiles");
  static_assert(kTG + kMaxPairs * kN2 <= (int)kTmemCols, "G accumulators in TMEM");
  static_assert(kN1 <= kTW && kD1Cols <= kTW, "P accumulators in TMEM");
  static_assert(kN2 % 16 == 0 && kN2 <= 256, "GEMM 2 shape");
  static_assert(kWs % 1024 == 0 && kPhiOff % 1024 == 0 && kWsOff % 1024 == 0, "swizzle alignment");
  static_assert(kXOff % 16 == 0 && kXBuf % 16 == 0, "exchange alignment");
  static_assert(kNumBars * 8 + 16 <= 512, "barrier area");
  static_assert(kSmemBytes <= kMaxSmem, "shared memory");
};

struct Args {
  int64_t n;
  int d[2];          // columns of the CTA's view (CCA: d_x, d_y; FDA: d, d)
  int pp[2];         // 128-column pairs of one part of each CTA
  int k2;            // columns of Phi (2k <= kXC)
  int D0;            // CCA: first G row of view 1 (d_x)
  int ntiles;
  const uint8_t* phi_img;  // [view][K-box][kN1 rows][128 B], pre-swizzled
  float* part;             // CCA: [cluster][D][4k]; FDA: [cluster][CTA][d][2k]
  int64_t slab;            // floats between partial slabs (a multiple of 4)
  int* err;
  const int* done;
  long long wait_limit;    // cycles of one pipeline wait before the kernel gives up
};

template <bool kLda>
__global__ void __launch_bounds__(256, 1)
split_pass_kernel(const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1,
                  const __grid_constant__ CUtensorMap tm2, const __grid_constant__ CUtensorMap tm3, Args a) {
  using L = SLay<kLda>;
  constexpr int kStages = L::kStages;
  if (a.done != nullptr && *a.done) return;  // uniform over the cluster: nothing remote has happened
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* ring = smem;
  uint8_t* phi_s = smem + L::kPhiOff;
  uint8_t* ws = smem + L::kWsOff;  // [buffer][hi | lo][kNW rows][128 B]
  float* xs = reinterpret_cast<float*>(smem + L::kXOff);  // [buffer][kRows][kXC]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOff);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + L::kNumBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cluster_ctarank();  // CCA: the view; FDA: 0 = hi part, 1 = lo part
  const uint32_t peer = 1u - (uint32_t)rank;
  const int cid = (int)cluster_id_x(), ncl = (int)cluster_count_x();
  const int view = kLda ? 0 : rank;
  const int pp = a.pp[rank];
  const int npairs = L::kParts * pp;
  const int split = (npairs + 1) / 2;  // GEMM 1: issuer 1 takes pairs [0, split), issuer 2 the rest
  const int nissue1 = split < npairs ? 2 : 1;
  const long long wl = a.wait_limit;
  auto bar = [&](int i) { return smem_u32(&bars[i]); };

  {
    uint4* wz = reinterpret_cast<uint4*>(ws);
    for (int i = threadIdx.x; i < 2 * L::kWBuf / 16; i += blockDim.x) wz[i] = make_uint4(0, 0, 0, 0);
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(bar(L::kFull + s), 1);
      mbar_init(bar(L::kEmpty + s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(L::kD1Full + b), nissue1);
      mbar_init(bar(L::kD1Free + b), 64);   // the two data warps
      mbar_init(bar(L::kXFull + b), 32);    // the peer's 32 row threads
      mbar_init(bar(L::kXFree + b), 2);     // the peer's two data warps
      mbar_init(bar(L::kWReady + b), 2);    // this CTA's two data warps
      mbar_init(bar(L::kWFree + b), 1);     // this CTA's GEMM 2 commit
    }
    mbar_init(bar(L::kGDone), 1);
    for (int i = 0; i < 3; ++i) mbar_init(bar(L::kFinal + i), 1);
    mbar_init(bar(L::kPhiFull), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers are initialised before any remote arrive
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int my_tiles = (a.ntiles - cid + ncl - 1) / ncl;
  const int nitems = my_tiles * npairs;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    bool ok = true;
    int last_use[kStages];
    for (int s = 0; s < kStages; ++s) last_use[s] = -1;
    const CUtensorMap* maps[2];
    if (kLda) {
      maps[0] = rank == 0 ? &tm0 : &tm1;
      maps[1] = maps[0];
    } else {
      maps[0] = rank == 0 ? &tm0 : &tm2;
      maps[1] = rank == 0 ? &tm1 : &tm3;
    }
    const int phi_bytes = 2 * pp * kKBox1;
    if (nitems > 0) {
      const uint32_t pb = bar(L::kPhiFull);
      mbar_expect_tx(pb, phi_bytes);
      for (int kb = 0; kb < 2 * pp; ++kb)
        bulk_g2s(smem_u32(phi_s + kb * kKBox1), a.phi_img + view * kPhiStride + kb * kKBox1, kKBox1, pb);
    }
    for (int it = 0; it < nitems; ++it) {
      const int j = it / npairs, p = it - j * npairs;
      const int part = p / pp, pl = p - part * pp;
      const int row0 = (cid + j * ncl) * kRows;
      const int slot = it % kStages, use = it / kStages;
      if (!mbar_wait(bar(L::kEmpty + slot), (use & 1) ^ 1, abort_flag, wl)) {
        ok = false;
        break;
      }
      const uint32_t fb = bar(L::kFull + slot);
      mbar_expect_tx(fb, kSlot);
      const uint32_t dst = smem_u32(ring + slot * kSlot);
      tma_load_2d(dst, maps[part], 128 * pl, row0, fb);
      tma_load_2d(dst + kBox, maps[part], 128 * pl + 64, row0, fb);
      last_use[slot] = use;
    }
    if (!ok) {
      // the copies this thread issued land before the CTA frees its memory
      if (nitems > 0) {
        const long long t0 = clock64();
        while (!mbar_try(bar(L::kPhiFull), 0) && clock64() - t0 < kWaitCycles) {
        }
      }
      for (int s = 0; s < kStages; ++s) {
        if (last_use[s] < 0) continue;
        const long long t0 = clock64();
        while (!mbar_try(bar(L::kFull + s), last_use[s] & 1) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if ((warp == 1 || warp == 3 || (warp == 2 && nissue1 == 2)) && lane == 0) {
    // ------------------------------------------------------------ MMA issuers
    constexpr uint32_t id1 = idesc_bf16(64, kN1, 0, 0);
    constexpr uint32_t id2 = idesc_bf16(128, L::kN2, 1, 0);
    bool ok = true;
    if (warp == 1 || warp == 2) {
      const int acc_i = warp - 1;
      const int pb = acc_i == 0 ? 0 : split, pe = acc_i == 0 ? split : npairs;
      const uint64_t bdesc0 = sdesc(smem_u32(phi_s), 16, 1024);
      if (my_tiles > 0) ok = mbar_wait(bar(L::kPhiFull), 0, abort_flag, wl);
      for (int j = 0; j < my_tiles && ok; ++j) {
        const int b = j & 1;
        if (j >= 2 && !(ok = mbar_wait(bar(L::kD1Free + b), ((j - 2) >> 1) & 1, abort_flag, wl))) break;
        tc_fence_after();
        const uint32_t d1 = tmem + (uint32_t)((2 * b + acc_i) * kTW);
        for (int p = pb; p < pe; ++p) {
          const int it = j * npairs + p;
          const int slot = it % kStages, use = it / kStages;
          const int pl = p % pp;
          if (!(ok = mbar_wait(bar(L::kFull + slot), use & 1, abort_flag, wl))) break;
          tc_fence_after();
          const uint64_t ad0 = sdesc(smem_u32(ring + slot * kSlot), 16, 1024);
          const uint64_t bd0 = bdesc0 + (uint64_t)((2 * pl * kKBox1) >> 4);
#define GB_S1_MMA(s, acc)                                                                   \
  mma_bf16(d1, ad0 + (uint64_t)((((s) >> 2) * kBox + ((s) & 3) * 32) >> 4),                 \
           bd0 + (uint64_t)((((s) >> 2) * kKBox1 + ((s) & 3) * 32) >> 4), id1, acc)
          if (p == pb) {
            GB_S1_MMA(0, 0u);
          } else {
            GB_S1_MMA(0, 1u);
          }
          GB_S1_MMA(1, 1u);
          GB_S1_MMA(2, 1u);
          GB_S1_MMA(3, 1u);
          GB_S1_MMA(4, 1u);
          GB_S1_MMA(5, 1u);
          GB_S1_MMA(6, 1u);
          GB_S1_MMA(7, 1u);
#undef GB_S1_MMA
        }
        if (!ok) break;
        mma_commit(bar(L::kD1Full + b));
      }
    } else {
      const uint64_t wd_base = sdesc(smem_u32(ws), 16, 1024);
      for (int j = 0; j < my_tiles && ok; ++j) {
        const int b = j & 1;
        if (!(ok = mbar_wait(bar(L::kWReady + b), (j >> 1) & 1, abort_flag, wl))) break;
        tc_fence_after();
        const uint64_t wd0 = wd_base + (uint64_t)((b * L::kWBuf) >> 4);
        for (int p = 0; p < npairs; ++p) {
          const int it = j * npairs + p;
          const int slot = it % kStages;
          const int pl = p % pp;
          const uint32_t g = tmem + (uint32_t)(L::kTG + pl * L::kN2);
          const uint64_t ad0 = sdesc(smem_u32(ring + slot * kSlot), kBox, 1024);
          // the hi and the lo part of the data accumulate into the same G
          const uint32_t acc0 = (j > 0 || p >= pp) ? 1u : 0u;
          mma_bf16(g, ad0, wd0, id2, acc0);
          mma_bf16(g, ad0 + (uint64_t)(2048 >> 4), wd0 + (uint64_t)(32 >> 4), id2, 1u);
          if (kLda) {  // the lo rows of W into the same accumulator
            const uint64_t wl0 = wd0 + (uint64_t)(L::kWs >> 4);
            mma_bf16(g, ad0, wl0, id2, 1u);
            mma_bf16(g, ad0 + (uint64_t)(2048 >> 4), wl0 + (uint64_t)(32 >> 4), id2, 1u);
          }
          mma_commit(bar(L::kEmpty + slot));
        }
        mma_commit(bar(L::kWFree + b));
      }
      if (ok) mma_commit(bar(L::kGDone));
    }
    if (!ok) {
      const int f = L::kFinal + (warp == 3 ? 1 : (warp == 2 ? 2 : 0));
      mma_commit(bar(f));
      const long long t0 = clock64();
      while (!mbar_try(bar(f), 0) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------ epilogue
    const int q = warp - 4;
    bool ok = true;
    if (q < 2) {
      // data warps: lanes 0..15 of warp q hold rows 16 q .. 16 q + 15 of the
      // tile (M = 64 layout: rows 16 q' .. 16 q' + 15 in lanes 32 q' ..)
      const uint32_t lane_off = (uint32_t)(32 * q) << 16;
      const int rr = 16 * q + (lane & 15);
      const bool upper = lane >= 16;
      for (int j = 0; j < my_tiles && ok; ++j) {
        const int b = j & 1;
        if (!(ok = mbar_wait(bar(L::kD1Full + b), (j >> 1) & 1, abort_flag, wl))) break;
        tc_fence_after();
        float d1[kD1Cols];
#pragma unroll
        for (int c = 0; c < kD1Cols; c += 16) tmem_ld16(tmem + lane_off + (uint32_t)(2 * b * kTW + c), &d1[c]);
        if (nissue1 == 2) {
          float d2[kD1Cols];
#pragma unroll
          for (int c = 0; c < kD1Cols; c += 16)
            tmem_ld16(tmem + lane_off + (uint32_t)((2 * b + 1) * kTW + c), &d2[c]);
          tmem_ld_wait();
#pragma unroll
          for (int c = 0; c < kD1Cols; ++c) d1[c] += d2[c];
        }
        tmem_ld_wait();
        tc_fence_before();
        mbar_arrive(bar(L::kD1Free + b));
        // own P row (the hi and lo columns of Phi added)
        float pw[kXC];
#pragma unroll
        for (int c = 0; c < kXC; ++c) pw[c] = d1[c] + d1[kH + c];
        // the peer has consumed the exchange buffer b of tile j - 2
        if (j >= 2 && !(ok = mbar_wait_cluster(bar(L::kXFree + b), ((j - 2) >> 1) & 1, abort_flag, wl))) break;
        if (!upper) {
          const uint32_t dst = map_peer(smem_u32(xs + (b * kRows + rr) * kXC), peer);
#pragma unroll
          for (int c = 0; c < kXC; c += 4) st_cluster_v4(dst + 4 * c, pw[c], pw[c + 1], pw[c + 2], pw[c + 3]);
          mbar_arrive_cluster(map_peer(bar(L::kXFull + b), peer));
        }
        // the peer's P row of this tile
        if (!(ok = mbar_wait_cluster(bar(L::kXFull + b), (j >> 1) & 1, abort_flag, wl))) break;
        // own row values for the upper lanes (same rows as lanes 0..15)
        float own[kXC];
#pragma unroll
        for (int c = 0; c < kXC; ++c) own[c] = __shfl_sync(0xffffffffu, pw[c], lane & 15);
        const float* pr = xs + (b * kRows + rr) * kXC;
        float oth[kXC];
#pragma unroll
        for (int c = 0; c < kXC; c += 4) {
          const float4 v = *reinterpret_cast<const float4*>(pr + c);
          oth[c] = v.x, oth[c + 1] = v.y, oth[c + 2] = v.z, oth[c + 3] = v.w;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(map_peer(bar(L::kXFree + b), peer));
        // this CTA's GEMM 2 of tile j - 2 is done with W buffer b
        if (j >= 2 && !(ok = mbar_wait(bar(L::kWFree + b), ((j - 2) >> 1) & 1, abort_flag, wl))) break;
        uint8_t* wb = ws + b * L::kWBuf;
        // W row rr: CCA [P_x | P_y] (lanes 0..15 write view 0's rows of the
        // operand, lanes 16..31 view 1's); FDA P_0 + P_1 (lanes 0..15 columns
        // 0..9, lanes 16..31 columns 10..19).  Then bf16 hi + lo; even lanes
        // store the pair of tile rows (rr, rr + 1), adjacent in the K-major
        // operand.
        constexpr int kNC = kLda ? kXC / 2 : kXC;  // columns per lane
        uint32_t hs[kNC], ls[kNC];
#pragma unroll
        for (int c0 = 0; c0 < kNC; ++c0) {
          float x;
          if (kLda) {
            const int c = upper ? c0 + kNC : c0;
            const float p0 = rank == 0 ? own[c] : oth[c];
            const float p1 = rank == 0 ? oth[c] : own[c];
            x = p0 + p1;
          } else {
            // view (upper ? 1 : 0): own if that is this CTA's view
            x = (upper ? 1 : 0) == rank ? own[c0] : oth[c0];
          }
          const __nv_bfloat16 hi = __float2bfloat16_rn(x);
          const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
          hs[c0] = __bfloat16_as_ushort(hi);
          ls[c0] = __bfloat16_as_ushort(lo);
        }
#pragma unroll
        for (int c0 = 0; c0 < kNC; ++c0) {
          hs[c0] |= __shfl_down_sync(0xffffffffu, hs[c0], 1) << 16;
          ls[c0] |= __shfl_down_sync(0xffffffffu, ls[c0], 1) << 16;
        }
        if ((lane & 1) == 0) {
#pragma unroll
          for (int c0 = 0; c0 < kNC; ++c0) {
            int orow, cc;
            if (kLda) {
              cc = upper ? c0 + kNC : c0;
              orow = cc;
            } else {
              cc = c0;
              orow = (upper ? kH : 0) + c0;
            }
            if (cc < a.k2) {
              const uint32_t off = swz(orow, rr);
              *reinterpret_cast<uint32_t*>(wb + off) = hs[c0];
              *reinterpret_cast<uint32_t*>(wb + L::kWs + off) = ls[c0];
            }
          }
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(L::kWReady + b));
      }
    }
    // ---------------------------------------------------- drain of G
    const uint32_t g_lane_off = (uint32_t)(32 * q) << 16;
    const int rg = 32 * q + lane;
    const int d = a.d[rank];
    float* out;
    int ostride;
    if (kLda) {
      out = a.part + ((int64_t)cid * 2 + rank) * a.slab;
      ostride = a.k2;
    } else {
      out = a.part + (int64_t)cid * a.slab + (int64_t)(rank == 0 ? 0 : a.D0) * 2 * a.k2;
      ostride = 2 * a.k2;
    }
    // every epilogue warp drains: the data warps' loop status and this
    // warp's own wait decide
    // (the warps without per-tile work wait here for the whole pass: their
    // bound is the default one, not the per-wait option)
    if (ok && my_tiles > 0 && !*abort_flag && mbar_wait(bar(L::kGDone), 0, abort_flag, q < 2 ? wl : kWaitCycles)) {
      tc_fence_after();
      for (int pl = 0; pl < pp; ++pl) {
        float g[L::kN2];
#pragma unroll
        for (int c = 0; c < L::kN2; c += 16) tmem_ld16(tmem + g_lane_off + (uint32_t)(L::kTG + pl * L::kN2 + c), &g[c]);
        tmem_ld_wait();
        const int col = 128 * pl + rg;
        if (col < d) {
          float* o = out + (int64_t)col * ostride;
          if (kLda) {
#pragma unroll
            for (int c = 0; c < kXC; ++c)
              if (c < a.k2) o[c] = g[c];
          } else {
#pragma unroll
            for (int c = 0; c < L::kNW; ++c) {
              const int vv = c / kH, cc = c - vv * kH;
              if (cc < a.k2) o[vv * a.k2 + cc] = g[c] + g[L::kNW + c];
            }
          }
        }
      }
    } else if (my_tiles > 0) {
      // a CTA that stopped early writes zeros (finite partials); the error
      // flag reports the failure
      for (int e = threadIdx.x - 128; e < d; e += 128)
        for (int c = 0; c < ostride; ++c) out[(int64_t)e * ostride + c] = 0.f;
    }
    tc_fence_before();
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicExch(a.err, kFlagTimeout);
  // all remote stores and arrives of both CTAs are complete after this
  // (release / acquire at cluster scope); nothing targets either CTA later
  cluster_sync();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Phi image for GEMM 1 (per view, K-boxes of 64 data columns; B rows
// 0 .. kH - 1 the bf16 hi parts of the 2k columns of Phi, rows kH .. 2 kH - 1
// their lo parts), 128B-swizzled; Phi rounded in place to hi + lo, the point
// the pass evaluates.  The image's padding is zero from its allocation.
__global__ void split_phi_image_kernel(double* __restrict__ Phix, double* __restrict__ Phiy, int dx, int dy,
                                       int k2, uint8_t* __restrict__ img) {
  const int v = blockIdx.y;
  const int d = v == 0 ? dx : dy;
  double* Phi = v == 0 ? Phix : Phiy;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d * k2) return;
  const int j = e / k2, c = e - j * k2;
  const double x = Phi[e];
  const __nv_bfloat16 hi = __double2bfloat16(x);
  const __nv_bfloat16 lo = __double2bfloat16(x - (double)__bfloat162float(hi));
  uint8_t* base = img + (int64_t)v * kPhiStride + (int64_t)(j >> 6) * kKBox1;
  *reinterpret_cast<__nv_bfloat16*>(base + swz(c, j & 63)) = hi;
  *reinterpret_cast<__nv_bfloat16*>(base + swz(kH + c, j & 63)) = lo;
  Phi[e] = (double)__bfloat162float(hi) + (double)__bfloat162float(lo);
}

// The BF16 hi / lo copy of an FP32 view (FDA: of its class-centred rows).
// Row i of the data goes to hi + i * hs and lo + i * hs (hs = row stride of
// the copy): separate hi and lo matrices (lo = hi + n ldo, hs = ldo), or rows
// interleaved (lo = hi + ldo, hs = 2 ldo: row 2i = hi, row 2i + 1 = lo).
__global__ void split_copy_kernel(const float* __restrict__ Z, int64_t ld, int64_t n, int d,
                                  const int32_t* __restrict__ y, const double* __restrict__ means,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t hs) {
  const int64_t total = n * (int64_t)d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / d;
    const int j = (int)(e - i * d);
    double v = (double)Z[i * ld + j];
    if (y != nullptr) v -= means[(int64_t)y[i] * d + j];
    const __nv_bfloat16 h = __double2bfloat16(v);
    hi[i * hs + j] = h;
    lo[i * hs + j] = __double2bfloat16(v - (double)__bfloat162float(h));
  }
}

// W^T W = Phi_bd^T G (nv views, nv k2 x nv k2) in FP64: one warp per entry.
__global__ void split_gram_kernel(const double* __restrict__ Phix, const double* __restrict__ Phiy, int dx, int dy,
                                  int k2, int nv, const double* __restrict__ G, double* __restrict__ Gram,
                                  const int* done) {
  if (done != nullptr && *done) return;
  const int nc = nv * k2;
  const int e = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (e >= nc * nc) return;
  const int ra = e / nc, cb = e - ra * nc;
  const int v = ra / k2;
  const int ca = ra - v * k2;
  const double* Phi = v == 0 ? Phix : Phiy;
  const int d = v == 0 ? dx : dy;
  const int off = v == 0 ? 0 : dx;
  double s = 0;
  for (int j = lane; j < d; j += 32) s += Phi[(int64_t)j * k2 + ca] * G[(int64_t)(off + j) * nc + cb];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) Gram[e] = s;
}

}  // namespace ts

// tc_reduce_kernel lives with the BF16 pass
namespace tc {
__global__ void tc_reduce_kernel(const float* __restrict__ part, int nparts, int64_t len, int64_t stride,
                                 double* __restrict__ G, const int* done, const int* nparts_dev, int ng, int col0,
                                 int k2);
}

// ----------------------------------------------------------------- host side
// FDA shapes of this kernel.  (CCA with FP32 data streams a row-interleaved
// copy through the BF16 kernel of pass_tc.cu, which shares the copy.)
bool split_pass_shape_ok(int kind, int dtype, int k, int d0, int d1) {
  if (dtype != GBCCA_FP32 || 2 * k > ts::kXC) return false;
  if (kind == kCCA) return false;
  (void)d1;
  return d0 <= 128 * ts::SLay<true>::kMaxPairs;
}

// CCA shapes of the interleaved copy for the BF16 kernel (any shape the
// library accepts: d <= 1024, k <= 20)
static bool interleaved_shape_ok(const Plan& p) { return p.kind == kCCA && p.dtype == GBCCA_FP32; }

bool split_pass_ready(const Plan& p) { return p.ts_img != nullptr && p.ts_ready && !p.ts_interleaved; }

int split_pass_alloc(Plan& p) {
  p.ts_ready = false;
  p.ts_interleaved = false;
  if (!p.opt.tensor_cores) return GBCCA_OK;
  if (interleaved_shape_ok(p)) {
    for (int v = 0; v < 2; ++v) {
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
    p.ts_interleaved = true;
    return GBCCA_OK;
  }
  if (!split_pass_shape_ok(p.kind, p.dtype, p.k, p.v[0].d, p.nviews > 1 ? p.v[1].d : 0)) return GBCCA_OK;
  for (int v = 0; v < p.nviews; ++v) {
    const int64_t ldo = (p.v[v].d + 7) / 8 * 8;
    p.ts_ld[v] = ldo;
    void* t = nullptr;  // the hi and the lo matrix, one after the other
    if (counted_malloc(&t, sizeof(__nv_bfloat16) * (size_t)2 * p.n * ldo) != cudaSuccess) {
      cudaGetLastError();
      set_last_error("allocation of the BF16 hi/lo copy of the data failed");
      return GBCCA_ERR_OOM;
    }
    p.ts_copy[v] = static_cast<__nv_bfloat16*>(t);
  }
  GB_CUDA(counted_malloc(reinterpret_cast<void**>(&p.ts_img), 2 * (size_t)ts::kPhiStride));
  GB_CUDA(cudaMemset(p.ts_img, 0, 2 * (size_t)ts::kPhiStride));
  // CCA: one slab of D x 4k per cluster; FDA: one of d x 2k per CTA; each
  // slab padded to a multiple of 4 floats (the reduction reads float4)
  const int64_t slab = ((int64_t)p.D * p.NC + 3) / 4 * 4;
  const int64_t slabs = p.kind == kCCA ? p.sm_count / 2 : 2 * (p.sm_count / 2);
  GB_CUDA(counted_malloc(reinterpret_cast<void**>(&p.ts_part), sizeof(float) * (size_t)std::max<int64_t>(1, slabs) * slab));
  return GBCCA_OK;
}

// Makes the BF16 hi/lo copies of the bound data (FDA: of the class-centred
// rows, after the class statistics) and their TMA descriptors.
int split_pass_prepare(Plan& p, cudaStream_t st) {
  p.ts_ready = false;
  if (!p.opt.tensor_cores || p.ts_copy[0] == nullptr) return GBCCA_OK;
  for (int v = 0; v < p.nviews; ++v) {
    const int d = p.v[v].d;
    const int64_t ldo = p.ts_ld[v];
    __nv_bfloat16* hi = p.ts_copy[v];
    __nv_bfloat16* lo = p.ts_interleaved ? hi + ldo : hi + p.n * ldo;
    const int64_t hs = p.ts_interleaved ? 2 * ldo : ldo;
    const int64_t total = p.n * (int64_t)d;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 8 * (int64_t)p.sm_count);
    ts::split_copy_kernel<<<grid, 256, 0, st>>>(static_cast<const float*>(p.v[v].Z), p.v[v].ld, p.n, d,
                                                p.kind == kLDA ? p.labels : nullptr,
                                                p.kind == kLDA ? p.means : nullptr, hi, lo, hs);
    GB_CHECK_LAUNCH();
    if (!p.ts_interleaved) {
      auto* m = reinterpret_cast<CUtensorMap*>(p.ts_map[2 * v]);
      GB_TRY(make_tma_map_bf16(m, hi, p.n, d, ldo, ts::kRows));
      GB_TRY(make_tma_map_bf16(m + 1, lo, p.n, d, ldo, ts::kRows));
    }
  }
  p.ts_ready = true;
  return GBCCA_OK;
}

int split_pass(Plan& p, cudaStream_t st, const int* done) {
  const bool lda = p.kind == kLDA;
  const int k2 = 2 * p.k;
  ts::Args a{};
  a.n = p.n;
  a.k2 = k2;
  if (lda) {
    a.d[0] = a.d[1] = p.v[0].d;
    a.pp[0] = a.pp[1] = ceil_div(p.v[0].d, 128);
    a.D0 = 0;
  } else {
    for (int v = 0; v < 2; ++v) {
      a.d[v] = p.v[v].d;
      a.pp[v] = ceil_div(p.v[v].d, 128);
    }
    a.D0 = p.v[0].d;
  }
  a.ntiles = ceil_div(p.n, ts::kRows);
  a.slab = ((int64_t)p.D * p.NC + 3) / 4 * 4;
  a.phi_img = p.ts_img;
  a.part = p.ts_part;
  a.err = p.flag;
  a.done = done;
  a.wait_limit = p.opt.wait_cycles > 0 ? p.opt.wait_cycles : tc::kWaitCycles;
  {
    const int dmax = std::max(p.v[0].d, p.nviews > 1 ? p.v[1].d : 0);
    ts::split_phi_image_kernel<<<dim3(ceil_div(dmax * k2, 256), p.nviews), 256, 0, st>>>(
        p.v[0].Phi, p.nviews > 1 ? p.v[1].Phi : p.v[0].Phi, p.v[0].d, p.nviews > 1 ? p.v[1].d : 0, k2, p.ts_img);
    GB_CHECK_LAUNCH();
  }
  auto kern = lda ? ts::split_pass_kernel<true> : ts::split_pass_kernel<false>;
  const int smem = lda ? ts::SLay<true>::kSmemBytes : ts::SLay<false>::kSmemBytes;
  GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (p.ts_clusters <= 0) {
    cfg.gridDim = dim3(2 * (p.sm_count / 2), 1, 1);
    int ncl = 0;
    GB_CUDA(cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg));
    p.ts_clusters = std::max(1, std::min(ncl, p.sm_count / 2));
  }
  const int ncl = std::min(p.ts_clusters, a.ntiles);
  cfg.gridDim = dim3(2 * ncl, 1, 1);
  const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(p.ts_map[0]);
  if (p.kev0 != nullptr) GB_CUDA(record_timing_event(p.kev0, st));
  GB_CUDA(cudaLaunchKernelEx(&cfg, kern, m[0], m[1], m[2], m[3], a));
  GB_CHECK_LAUNCH();
  if (p.kev1 != nullptr) GB_CUDA(record_timing_event(p.kev1, st));
  const int nparts = lda ? 2 * ncl : ncl;
  const int64_t len = (int64_t)p.D * p.NC;
  tc::tc_reduce_kernel<<<ceil_div(len, 256), 256, 0, st>>>(p.ts_part, nparts, len, a.slab, p.G, done, nullptr,
                                                           0, 0, 0);
  GB_CHECK_LAUNCH();
  const int nc = p.NC;
  ts::split_gram_kernel<<<ceil_div((int64_t)nc * nc * 32, 256), 256, 0, st>>>(
      p.v[0].Phi, p.nviews > 1 ? p.v[1].Phi : nullptr, p.v[0].d, p.nviews > 1 ? p.v[1].d : 0, k2, p.nviews, p.G,
      p.Gram, done);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

}  // namespace gbcca
