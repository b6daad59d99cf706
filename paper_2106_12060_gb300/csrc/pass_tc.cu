// Tensor-core (tcgen05 + TMA) fused CCA data pass for BF16 data on sm_103a,
// and for FP32 data streamed as a row-interleaved BF16 hi/lo copy (row 2i =
// bf16(z_i), row 2i + 1 = bf16(z_i - bf16(z_i)); see `pair_sum`).  The FDA
// pass (Sec. 5.1-5.2, Cor. 5.6: S_w Phi = Xhat^T (Xhat Phi) over the copy of
// the class-centred rows) is the same kernel in one-view clusters (kSolo):
// both CTAs stream the one view, each half of its 128-column pairs, and add
// their partial products W of every tile before GEMM 2.
//
// One Riemannian-CG iteration of the CCA solver needs, for the block-diagonal
// Phi = blkdiag([U, eta_U], [V, eta_V]) (Sec. 4.2 gradient, Table 1
// retraction, Cor. 4.6 per-iteration cost O(p (nnz X + nnz Y))):
//     W = Z Phi  (Z = [X | Y], n x 4k, never leaves the chip)
//     G = Z^T W  (D x 4k)
// and W^T W, which equals Phi^T G and is formed afterwards in FP64 from G.
//
// Persistent kernel of 2-CTA clusters; both CTAs of a cluster work on the
// same 64-row tile, CTA v on view v (X or Y), so that each CTA keeps its
// 64 x d_v BF16 block (<= 64 KB) in shared memory for both GEMMs and every
// byte of the data is read from HBM exactly once.  Two tiles are resident per
// CTA (double buffering): the next tile streams in while the current one is
// in its epilogue and second GEMM.  Per tile (h = 20 for 2k <= 20, else 24):
//   GEMM 1  (tcgen05, M = 64, per CTA): W_v = Z_v Phi_v, 64 x 2h FP32 in TMEM
//           (B = Phi_v split into bf16 hi|lo columns, h each; rows 16 q ..
//           16 q + 15 of the M = 64 result sit in lanes 32 q .. 32 q + 15);
//   epilogue warps read W_v from TMEM, add the hi and lo halves, split W_v
//           into bf16 hi/lo and write it into the K-major B operand of GEMM 2
//           (rows h v .. h v + h - 1 of the hi part and of the lo part) of
//           their own CTA, then push those rows into the peer CTA's operand
//           with bulk shared::cluster copies;
//   GEMM 2  (tcgen05, M = 128, N = 4h, per CTA): G_v += Z_v^T [W_x | W_y]
//           for the hi and the lo parts at once (separate accumulator
//           columns, added when G is drained), over the same shared-memory
//           blocks read as MN-major A (128 columns of Z_v per MMA),
//           accumulated in TMEM over all tiles of the cluster.  One MMA per
//           K step reads each block of the tile once: the operand reads from
//           shared memory, not the tensor arithmetic, bound these small-N
//           products.
// The end of GEMM 2 is signalled to both CTAs (multicast commit), which
// frees both CTAs' W operand buffer of that tile.  At the end the epilogue
// warps drain G to a per-cluster FP32 partial; a second kernel sums the
// partials in fixed order.
//
// Roles per CTA: warp 0 lane 0 = TMA producer (it first issues the bulk copy
// of the own view's Phi image, so the ring starts filling at once); warp 1
// lane 0 = GEMM 1 issuer (with 2k <= 20: for the first half of the pairs,
// warp 2 lane 0 for the second half, into a second accumulator that the
// epilogue adds); warp 3 lane 0 = GEMM 2 issuer; warp 2 = TMEM allocator;
// warps 4-7 and 8-11 = two epilogue groups (even and odd tiles; TMEM lane
// quarters 0-3 each), whose per-tile chains of dependent steps overlap.
// Every mbarrier wait is bounded in time; on expiry the CTA records an error
// code, waits (bounded) for its own copies and MMAs, frees TMEM and leaves
// after a cluster barrier (no remote access can target an exited CTA).
#include <cstring>
#include <vector>

#include "tc_ptx.cuh"

namespace gbcca {

namespace tc {

constexpr int kRows = 64;             // rows per tile (MMA M of GEMM 1, K of GEMM 2)
constexpr int kHalfMax = 24;          // W rows of a view at most (2k <= 24)
constexpr int kTileSlots = 4;         // pair slots of one tile (512 columns)
constexpr int kSlot = 16384;          // two 64 x 64 BF16 boxes
constexpr int kBox = 8192;
constexpr int kPhiView = 49152;       // stride of the views' Phi images in the plan buffer
constexpr int kMaxSmem = 232448;      // dynamic shared memory of one CTA
constexpr uint32_t kTmemCols = 512;   // W: columns kTW (nacc b + a); G: kTG + kN2 p (p < 4 pairs)
constexpr int kTW = 48;               // TMEM column stride of the W accumulators
constexpr long long kTimeout = kWaitCycles;       // cycles (~1 s)

// Shared-memory layout and barriers for GEMM 1 with N = 2 kH1 (Phi columns as
// bf16 hi rows 0 .. kH1 - 1 and lo rows kH1 .. 2 kH1 - 1; kH1 = 20 serves
// 2k <= 20 and leaves room for a 10-slot ring, kH1 = 24 a 9-slot ring).
template <int kH1, bool kQuad = false, bool kSolo = false>
struct Lay {
  static constexpr int kN1 = 2 * kH1;
  static constexpr int kKBox1 = kN1 * 128;       // one K-box (64 columns) of the Phi image
  static constexpr int kPhiBytes = 8 * kKBox1;   // 512 columns
  // W operand of GEMM 2 (K-major, one K-box of 64 tile rows): rows
  // [W_x | W_y] of the hi parts (kH1 rows per view; rows 2k .. kH1 - 1 stay
  // zero), then the same rows of the lo parts, so that one MMA with
  // N = kN2 reads the tile's columns once for both parts.  One view (FDA):
  // its rows padded to 24 per part (an M = 128 MMA needs N a multiple of 16).
  static constexpr int kHalf = kH1;              // W rows of a view
  static constexpr int kNW = kSolo ? 24 : 2 * kH1;  // rows of one part (hi or lo)
  static constexpr int kN2 = 2 * kNW;            // N of GEMM 2
  static constexpr int kWs = kNW * 128;          // bytes of one part
  static constexpr int kWBuf = 2 * kWs;          // hi + lo
  static constexpr int kWHalf = kHalf * 128;     // one view's rows of one part
  static constexpr int kD1Cols = ((kN1 + 15) / 16) * 16;  // TMEM columns read back for W
  // GEMM 1 is issued by two threads (pairs [0, ceil(np / 2)) and the rest),
  // each into its own accumulator, when TMEM has room for 2 x 2 W
  // accumulators and the G accumulators: one thread issues an MMA only about
  // every 50 cycles, two streams overlap in the tensor pipe.
  static constexpr int kNAcc = (4 * kTW + kTileSlots * kN2 <= (int)kTmemCols) ? 2 : 1;
  static constexpr int kTG = 2 * kNAcc * kTW;    // first TMEM column of the G accumulators
  // 4-CTA clusters (views wider than 512 columns, split over two CTAs each)
  // and one-view clusters (FDA: the view's columns split over the two CTAs):
  // two FP32 buffers that receive the other half's partial W of a tile
  static constexpr bool kHalves = kQuad || kSolo;  // a view's pairs over two CTAs
  static constexpr int kXC = 24;                 // floats per row of an exchange buffer
  static constexpr int kXBytes = kHalves ? 2 * kRows * kXC * 4 : 0;
  static constexpr int kStages = (kMaxSmem - kPhiBytes - 2 * kWBuf - kXBytes - 512 - 1024) / kSlot;
  static constexpr int kRingOff = kPhiBytes;
  static constexpr int kWsOff = kRingOff + kStages * kSlot;
  static constexpr int kXOff = kWsOff + 2 * kWBuf;
  static constexpr int kBarOff = kXOff + kXBytes;
  static constexpr int kSmemBytes = kBarOff + 512 + 1024;  // barriers + alignment slack
  // barrier indices
  static constexpr int kFull = 0, kEmpty = kStages, kD1Full = 2 * kStages;  // [stages], [stages], [2]
  static constexpr int kD1Free = kD1Full + 2, kEpiSync = kD1Free + 2, kWReady = kEpiSync + 1;  // [2], 1, [2]
  static constexpr int kWPeer = kWReady + 2, kWFree = kWPeer + 2, kGDone = kWFree + 2;      // [2], [2], 1
  static constexpr int kFinal = kGDone + 1;                         // [3]: one per MMA-issuing thread
  static constexpr int kPhiFull = kFinal + 3;  // Phi image in shared memory
  static constexpr int kGFree = kPhiFull + 1;   // G drained (128 arrivals)
  static constexpr int kPhiFree = kGFree + 1;  // GEMM 1 done with a segment's Phi
  static constexpr int kXFull = kPhiFree + 1, kXFree = kXFull + 2;  // [2], [2]: partial-W exchange (quad)
  static constexpr int kEpiSyncB = kXFree + 2;  // the second epilogue group's kEpiSync
  static constexpr int kNumBars = kEpiSyncB + 1;
  static_assert(!(kQuad && kSolo), "one cluster shape");
  static_assert(kStages >= 2 * kTileSlots, "two resident tiles");
  static_assert(kN1 <= kTW && kD1Cols <= kTW, "W buffers in TMEM");
  static_assert(kN2 % 16 == 0 && kTG + kTileSlots * kN2 <= (int)kTmemCols, "G accumulators in TMEM");
  static_assert(kPhiBytes % 16 == 0 && kWHalf % 16 == 0 && kWs % 1024 == 0, "bulk copy and swizzle alignment");
  static_assert(kRows == 64, "GEMM 2 issues four K steps of 16 rows");
  static_assert(kNumBars * 8 + 8 <= 512, "barrier area");
  static_assert(kSmemBytes <= kMaxSmem, "shared memory");
};

// One instance of a batched pass (device memory; the tensor maps are read by
// the TMA unit from there; CUtensorMap carries its own 128-byte alignment).
struct Inst {
  CUtensorMap map[2];      // views X, Y (BF16 data, or the interleaved hi/lo copy)
  const uint8_t* phi_img;  // [view][K-box][2 kH1][128 B], pre-swizzled
  float* partG;            // [slab][D][4k] partials of this instance
  const int* done;         // the instance's convergence flag: skip it when set
  int64_t slab;            // floats per partial slab (D * 4k)
  int64_t img_view;        // bytes between the two views' Phi images
  int d[2];
  int pairs[2];
  int k2;
  int pair_sum;
};

// A contiguous range of one instance's 64-row tiles, processed by one cluster
// into partial slab `slab` of that instance.
struct Seg {
  int inst;
  int first;
  int count;
  int slab;
};

struct Args {
  // one instance (insts == nullptr): cluster c takes tiles c, c + clusters,
  // ... of the pair of matrices in the kernel's tensor-map parameters
  int64_t n;
  int d[2];
  int pairs[2];
  int k2;        // columns of Phi per view (2k)
  int ntiles;
  const uint8_t* phi_img;  // [view][K-box][2 kH1][128 B], pre-swizzled
  float* partG;            // [cluster][D][4k] (one view: [cluster][d][2k])
  int64_t slab;            // floats between the clusters' partial slabs (a multiple of 4)
  int* err;
  const int* done;
  int64_t img_view;        // bytes between the two views' Phi images
  int pair_sum;            // 1: rows 2i and 2i+1 of the streamed matrix are the bf16
                           // hi and lo parts of one data row (FP32 data): W of the
                           // row is the sum of the two product rows, and both rows
                           // of GEMM 2's operand carry it
  long long wait_limit;    // one-view clusters: cycles of one pipeline wait before the
                           // kernel gives up (the other shapes use kWaitCycles)
  // several instances (insts != nullptr): cluster c takes the segments
  // seg_off[c] .. seg_off[c + 1] - 1 in order
  const Inst* insts;
  const Seg* segs;
  const int* seg_off;      // [clusters + 1]
};

// What one CTA needs of the segment it is on.
struct SegView {
  const CUtensorMap* map;  // this CTA's view
  const uint8_t* phi;      // this view's Phi image
  float* out;              // partial slab of the segment
  int first, stride, count;
  int d0, d1, npairs, k2, pair_sum;
  int pb;                  // first 128-column pair of this CTA (4-CTA clusters: half h of the view)
  bool skip;
};

// The 128-column pairs of a view of P pairs that CTA half h takes: all of
// them in a 2-CTA cluster of two views; in a 4-CTA cluster, or a one-view
// cluster, the first ceil(P / 2) for h = 0 and the rest for h = 1, at least
// one (a pair past the view's last column reads zeros from the tensor map and
// the image, and drains nothing).
__device__ __forceinline__ void half_pairs(int P, bool split, int h, int* pb, int* np) {
  if (!split) {
    *pb = 0;
    *np = P;
    return;
  }
  const int p0 = (P + 1) / 2;
  *pb = h == 0 ? 0 : p0;
  *np = h == 0 ? p0 : max(1, P - p0);
}

__device__ __forceinline__ int seg_count(const Args& a, int cid, int ncl) {
  if (a.insts == nullptr) return 1;
  return a.seg_off[cid + 1] - a.seg_off[cid];
}

// (split: the view's pairs are split over two CTAs)
__device__ __forceinline__ SegView seg_view(const Args& a, const CUtensorMap* tmx, const CUtensorMap* tmy, int view,
                                            int cid, int ncl, int s, bool split = false, int half = 0) {
  SegView v;
  if (a.insts == nullptr) {
    v.map = view == 0 ? tmx : tmy;
    v.phi = a.phi_img + view * a.img_view;
    v.d0 = a.d[0];
    v.d1 = a.d[1];
    v.out = a.partG + (int64_t)cid * a.slab;
    v.first = cid;
    v.stride = ncl;
    v.count = (a.ntiles - cid + ncl - 1) / ncl;
    half_pairs(a.pairs[view], split, half, &v.pb, &v.npairs);
    v.k2 = a.k2;
    v.pair_sum = a.pair_sum;
    v.skip = false;
  } else {
    const Seg sg = a.segs[a.seg_off[cid] + s];
    const Inst* I = a.insts + sg.inst;
    v.map = &I->map[view];
    v.phi = I->phi_img + view * I->img_view;
    v.out = I->partG + (int64_t)sg.slab * I->slab;
    v.d0 = I->d[0];
    v.d1 = I->d[1];
    v.first = sg.first;
    v.stride = 1;
    v.count = sg.count;
    half_pairs(I->pairs[view], split, half, &v.pb, &v.npairs);
    v.k2 = I->k2;
    v.pair_sum = I->pair_sum;
    v.skip = I->done != nullptr && *I->done != 0;
  }
  if (v.skip) v.count = 0;
  return v;
}

constexpr int kThreads = 384;  // 4 role warps + two epilogue groups of 4 warps

template <int kH1, bool kQuad = false, bool kSolo = false>
__global__ void __launch_bounds__(kThreads, 1)
tc_pass_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmy, Args a) {
  using L = Lay<kH1, kQuad, kSolo>;
  constexpr bool kHalves = L::kHalves;
  constexpr int kNvs = kSolo ? 1 : 2;  // views per row of a partial slab
  constexpr int kStages = L::kStages;
  constexpr int kFull = L::kFull, kEmpty = L::kEmpty, kD1Full = L::kD1Full, kD1Free = L::kD1Free;
  constexpr int kEpiSync = L::kEpiSync, kWReady = L::kWReady, kWPeer = L::kWPeer, kWFree = L::kWFree;
  constexpr int kGDone = L::kGDone, kFinal = L::kFinal, kPhiFull = L::kPhiFull, kGFree = L::kGFree;
  constexpr int kPhiFree = L::kPhiFree, kXFull = L::kXFull, kXFree = L::kXFree, kEpiSyncB = L::kEpiSyncB;
  constexpr int kNumBars = L::kNumBars;
  constexpr int kTG = L::kTG;
  if (a.done != nullptr && *a.done) return;  // uniform over the cluster: no remote access yet
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* phi_s = smem;
  uint8_t* ring = smem + L::kRingOff;
  uint8_t* ws = smem + L::kWsOff;  // [buffer][hi | lo][kNW rows][128 B]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOff);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kNumBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* xbuf = reinterpret_cast<float*>(smem + L::kXOff);  // [buffer][64 rows][kXC]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // rank = 2 half + view: CTAs 2h and 2h + 1 form the pair that shares the
  // tile's W (views X and Y); in a 4-CTA cluster, CTAs v and v + 2 hold the
  // two column halves of view v and add their partial W of every tile.  A
  // one-view cluster (FDA): rank = half, the two CTAs add their partial W.
  const uint32_t rank = cluster_ctarank();
  const int view = kSolo ? 0 : (int)(rank & 1u);  // 0: X, 1: Y
  const int half = kQuad ? (int)(rank >> 1) : (kSolo ? (int)rank : 0);
  const uint32_t peer = rank ^ 1u;
  const uint32_t hpeer = kSolo ? rank ^ 1u : rank ^ 2u;
  (void)hpeer;
  (void)xbuf;
  // bound of one pipeline wait: the plan's for a one-view cluster, whose only
  // remote operations are synchronous stores and arrivals (an abort leaves no
  // copy in flight towards the peer); the default otherwise
  const long long wl = kSolo ? a.wait_limit : kWaitCycles;
  const int cid = (int)cluster_id_x(), ncl = (int)cluster_count_x();
  const int nseg = seg_count(a, cid, ncl);
  auto bar = [&](int i) { return smem_u32(&bars[i]); };

  // zero the W operands (each view's Phi image arrives by bulk copies that
  // the producer issues ahead of the first tile of each segment)
  {
    uint4* wz = reinterpret_cast<uint4*>(ws);
    for (int i = threadIdx.x; i < 2 * L::kWBuf / 16; i += blockDim.x) wz[i] = make_uint4(0, 0, 0, 0);
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(bar(kFull + s), 1);
      mbar_init(bar(kEmpty + s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(kD1Full + b), L::kNAcc);  // one arrival per GEMM 1 issuer
      mbar_init(bar(kD1Free + b), 128);
      mbar_init(bar(kWReady + b), 1);
      mbar_init(bar(kWPeer + b), 1);   // + the peer's bytes
      mbar_init(bar(kWFree + b), kSolo ? 1 : 2);  // own (and the peer's) end of GEMM 2
    }
    mbar_init(bar(kEpiSync), 128);
    mbar_init(bar(kEpiSyncB), 128);
    mbar_init(bar(kGDone), 1);
    mbar_init(bar(kGFree), 128);
    mbar_init(bar(kPhiFree), L::kNAcc);  // one arrival per GEMM 1 issuer
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(kXFull + b), 4);  // the other half's epilogue warps
      mbar_init(bar(kXFree + b), 4);
    }
    mbar_init(bar(kFinal), 1);
    mbar_init(bar(kFinal + 1), 1);
    mbar_init(bar(kFinal + 2), 1);
    mbar_init(bar(kPhiFull), 1);
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
  cluster_sync();  // both CTAs' barriers and W operands are initialised
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // Every role walks the same segments and tiles; jg counts the tiles and ig
  // the (tile, pair) items this CTA has processed (barrier phases and ring
  // slots run on across segments), sp the segments with tiles.
  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    bool ok = true;
    int last_use[kStages];
    for (int s = 0; s < kStages; ++s) last_use[s] = -1;
    int jg = 0, ig = 0, sp = 0;
    for (int s = 0; s < nseg && ok; ++s) {
      const SegView sv = seg_view(a, &tmx, &tmy, view, cid, ncl, s, kHalves, half);
      if (sv.count == 0) continue;
      // the Phi image is rewritten only after every GEMM 1 MMA of the
      // previous segment has completed (its issuers signal that once per
      // segment; the barrier of a tile could already be two phases behind
      // this thread, whose parity test would then pass too early)
      if (sp > 0 && !(ok = mbar_wait(bar(kPhiFree), (sp - 1) & 1, abort_flag, wl))) break;
      // this segment's Phi image (GEMM 1's B operand), one bulk copy per K-box
      const uint32_t pb = bar(kPhiFull);
      mbar_expect_tx(pb, L::kPhiBytes);
      // (this CTA's pairs: K-boxes 2 pb .. 2 pb + 7 of the image)
      for (int kb = 0; kb < 8; ++kb)
        bulk_g2s(smem_u32(phi_s + kb * L::kKBox1), sv.phi + (2 * sv.pb + kb) * L::kKBox1, L::kKBox1, pb);
      ++sp;
      for (int t = 0; t < sv.count && ok; ++t, ++jg) {
        const int row0 = (sv.first + t * sv.stride) * kRows;
        for (int p = 0; p < sv.npairs; ++p, ++ig) {
          const int slot = ig % kStages, use = ig / kStages;
          if (!(ok = mbar_wait(bar(kEmpty + slot), (use & 1) ^ 1, abort_flag, wl))) break;
          const uint32_t fb = bar(kFull + slot);
          mbar_expect_tx(fb, kSlot);
          const uint32_t dst = smem_u32(ring + slot * kSlot);
          tma_load_2d(dst, sv.map, 128 * (sv.pb + p), row0, fb);
          tma_load_2d(dst + kBox, sv.map, 128 * (sv.pb + p) + 64, row0, fb);
          last_use[slot] = use;
        }
      }
    }
    if (!ok) {
      // wait (bounded) for the copies this thread issued before leaving
      if (sp > 0) {
        const long long t0 = clock64();
        while (!mbar_try(bar(kPhiFull), (sp - 1) & 1) && clock64() - t0 < kTimeout) {
        }
      }
      for (int s = 0; s < kStages; ++s) {
        if (last_use[s] < 0) continue;
        const long long t0 = clock64();
        while (!mbar_try(bar(kFull + s), last_use[s] & 1) && clock64() - t0 < kTimeout) {
        }
      }
    }
  } else if ((warp == 1 || warp == 3 || (warp == 2 && L::kNAcc == 2)) && lane == 0) {
    // ------------------------------------------------------------ MMA issuers
    // warps 1 and 2: GEMM 1 of every tile (half of the pairs each when there
    // are two accumulators); warp 3: GEMM 2 of every tile.  Separate issuers
    // keep GEMM 2 of tile j (which frees its ring slots) from waiting behind
    // the arrival of tile j + 1's data.
    constexpr uint32_t id1 = idesc_bf16(64, L::kN1, 0, 0);
    constexpr uint32_t id2 = idesc_bf16(128, L::kN2, 1, 0);
    bool ok = true;
    int issued = 0;  // MMAs this thread has issued
    int jg = 0, ig = 0, sp = 0;
    // One thread issues an MMA only about every 50 cycles at best, which for
    // these small shapes is slower than the tensor pipe; the issue loops
    // therefore do no descriptor arithmetic beyond one add of a compile-time
    // offset (a descriptor's low bits are the shared-memory address / 16,
    // and every operand address here is below 2^18).
    if (warp == 1 || warp == 2) {
      const int acc_i = warp - 1;  // accumulator of this issuer
      const uint64_t bdesc0 = sdesc(smem_u32(phi_s), 16, 1024);
      for (int s = 0; s < nseg && ok; ++s) {
        const SegView sv = seg_view(a, &tmx, &tmy, view, cid, ncl, s, kHalves, half);
        if (sv.count == 0) continue;
        const int npairs = sv.npairs;
        const int split = L::kNAcc == 2 ? (npairs + 1) / 2 : npairs;
        const int pb = acc_i == 0 ? 0 : split, pe = acc_i == 0 ? split : npairs;
        if (!(ok = mbar_wait(bar(kPhiFull), sp & 1, abort_flag, wl))) break;
        ++sp;
        for (int t = 0; t < sv.count && ok; ++t, ++jg, ig += npairs) {
          const int b = jg & 1;
          // W buffer b was last read by the epilogue of tile jg - 2
          if (jg >= 2 && !(ok = mbar_wait(bar(kD1Free + b), ((jg - 2) >> 1) & 1, abort_flag, wl))) break;
          tc_fence_after();
          const uint32_t d1 = tmem + (uint32_t)((L::kNAcc * b + acc_i) * kTW);
          for (int p = pb; p < pe; ++p) {
            const int it = ig + p;
            const int slot = it % kStages, use = it / kStages;
            if (!(ok = mbar_wait(bar(kFull + slot), use & 1, abort_flag, wl))) break;
            tc_fence_after();
            const uint64_t ad0 = sdesc(smem_u32(ring + slot * kSlot), 16, 1024);
            const uint64_t bd0 = bdesc0 + (uint64_t)((2 * p * L::kKBox1) >> 4);
            // K steps of 16 columns: box s / 4 of the slot, 32-byte step s % 4
            // inside its 128-byte swizzled rows
#define GB_G1_MMA(s, acc)                                                                        \
  mma_bf16(d1, ad0 + (uint64_t)((((s) >> 2) * kBox + ((s) & 3) * 32) >> 4),                      \
           bd0 + (uint64_t)((((s) >> 2) * L::kKBox1 + ((s) & 3) * 32) >> 4), id1, acc)
            if (p == pb) {
              GB_G1_MMA(0, 0u);
            } else {
              GB_G1_MMA(0, 1u);
            }
            GB_G1_MMA(1, 1u);
            GB_G1_MMA(2, 1u);
            GB_G1_MMA(3, 1u);
            GB_G1_MMA(4, 1u);
            GB_G1_MMA(5, 1u);
            GB_G1_MMA(6, 1u);
            GB_G1_MMA(7, 1u);
#undef GB_G1_MMA
            issued += 8;
          }
          if (!ok) break;
          // an issuer without pairs in this segment arrives plainly; the
          // barrier then completes with the other issuer's MMAs
          if (pe > pb) {
            mma_commit(bar(kD1Full + b));
          } else {
            mbar_arrive(bar(kD1Full + b));
          }
        }
        if (!ok) break;
        // release the Phi image when a later segment will load its own
        bool more = false;
        for (int s2 = s + 1; s2 < nseg && !more; ++s2)
          more = seg_view(a, &tmx, &tmy, view, cid, ncl, s2, kHalves, half).count > 0;
        if (more) {
          if (pe > pb) {
            mma_commit(bar(kPhiFree));
          } else {
            mbar_arrive(bar(kPhiFree));
          }
        }
      }
    } else {
      for (int s = 0; s < nseg && ok; ++s) {
        const SegView sv = seg_view(a, &tmx, &tmy, view, cid, ncl, s, kHalves, half);
        if (sv.count == 0) continue;
        const int npairs = sv.npairs;
        // the epilogue has drained the G accumulators of the previous segment
        if (sp > 0 && !(ok = mbar_wait(bar(kGFree), (sp - 1) & 1, abort_flag, wl))) break;
        tc_fence_after();
        ++sp;
        for (int t = 0; t < sv.count && ok; ++t, ++jg, ig += npairs) {
          const int b = jg & 1;
          // both halves of this tile's W operand: ours and the peer's (one
          // view: ours alone)
          if (!kSolo) mbar_expect_tx(bar(kWPeer + b), 2 * L::kWHalf);
          if (!(ok = mbar_wait(bar(kWReady + b), (jg >> 1) & 1, abort_flag, wl))) break;
          if (!kSolo && !(ok = mbar_wait(bar(kWPeer + b), (jg >> 1) & 1, abort_flag, wl))) break;
          tc_fence_after();
          const uint64_t wd0 = sdesc(smem_u32(ws + b * L::kWBuf), 16, 1024);
          const uint32_t acc0 = t > 0 ? 1u : 0u;
          for (int p = 0; p < npairs; ++p) {
            const int it = ig + p;
            const int slot = it % kStages;
            const uint32_t g = tmem + (uint32_t)(kTG + p * L::kN2);
            const uint64_t ad0 = sdesc(smem_u32(ring + slot * kSlot), kBox, 1024);
            // B = the hi rows and then the lo rows of W (N = kN2): the tile's
            // columns are read once per K step of 16 rows (A: 8-row groups of
            // 1024 bytes, B: 32-byte steps inside the swizzled rows); the lo
            // products accumulate in their own columns of G
            mma_bf16(g, ad0, wd0, id2, acc0);
            mma_bf16(g, ad0 + (uint64_t)(2048 >> 4), wd0 + (uint64_t)(32 >> 4), id2, 1u);
            mma_bf16(g, ad0 + (uint64_t)(4096 >> 4), wd0 + (uint64_t)(64 >> 4), id2, 1u);
            mma_bf16(g, ad0 + (uint64_t)(6144 >> 4), wd0 + (uint64_t)(96 >> 4), id2, 1u);
            mma_commit(bar(kEmpty + slot));
            issued += 4;
          }
          // both CTAs learn that this CTA's GEMM 2 has consumed buffer b (one
          // view: this CTA alone reads its W operand)
          if constexpr (kSolo) {
            mma_commit(bar(kWFree + b));
          } else {
            mma_commit_mc(bar(kWFree + b), (uint16_t)(0x3u << (2 * half)));
          }
        }
        if (ok) mma_commit(bar(kGDone));  // this segment's G is complete
      }
    }
    if (!ok && issued > 0) {
      // let the MMAs this thread issued finish before the CTA frees its memory
      const int f = kFinal + (warp == 3 ? 1 : (warp == 2 ? 2 : 0));
      mma_commit(bar(f));
      const long long t0 = clock64();
      while (!mbar_try(bar(f), 0) && clock64() - t0 < kTimeout) {
      }
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------ epilogue
    // Two groups of four warps: group g takes the tiles jg with jg % 2 == g
    // (their W and GEMM 1 accumulator buffer g), so that the epilogues of
    // two consecutive tiles run at once; group 0 drains G at segment ends.
    const int grp = (warp - 4) >> 2;
    const int q = warp & 3;             // TMEM lane quarter (a warp reaches lanes 32 (warp % 4) ..)
    const int esync = grp == 0 ? kEpiSync : kEpiSyncB;
    const int lead = 128 * (grp + 1);   // the group's first thread
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    const int rg = 32 * q + lane;       // Z column of a G pair block (M = 128 layout)
    bool ok = true;
    int jg = 0, sp = 0;
    for (int s = 0; s < nseg && ok; ++s) {
      const SegView sv = seg_view(a, &tmx, &tmy, view, cid, ncl, s, kHalves, half);
      if (sv.count == 0) continue;
      const int npairs = sv.npairs;
      const bool two_acc = L::kNAcc == 2 && (npairs + 1) / 2 < npairs;
      for (int t = 0; t < sv.count; ++t, ++jg) {
        const int b = jg & 1;
        if (b != grp) continue;
        if (!(ok = mbar_wait(bar(kD1Full + b), (jg >> 1) & 1, abort_flag, wl))) break;
        tc_fence_after();
        float d1[L::kD1Cols];
#pragma unroll
        for (int c = 0; c < L::kD1Cols; c += 16)
          tmem_ld16(tmem + lane_off + (uint32_t)(L::kNAcc * b * kTW + c), &d1[c]);
        if (two_acc) {
          // second GEMM 1 accumulator (the other half of the pairs)
          float d2[L::kD1Cols];
#pragma unroll
          for (int c = 0; c < L::kD1Cols; c += 16)
            tmem_ld16(tmem + lane_off + (uint32_t)((L::kNAcc * b + 1) * kTW + c), &d2[c]);
          tmem_ld_wait();
#pragma unroll
          for (int c = 0; c < L::kD1Cols; ++c) d1[c] += d2[c];
        }
        tmem_ld_wait();
        tc_fence_before();
        mbar_arrive(bar(kD1Free + b));
        // both CTAs' GEMM 2 of tile jg - 2 must be done with both halves of buffer b
        if (jg >= 2 && !(ok = mbar_wait(bar(kWFree + b), ((jg - 2) >> 1) & 1, abort_flag, wl))) break;
        uint8_t* wb = ws + b * L::kWBuf;
        {
          // W_v row rr = hi part (TMEM column c) + lo part (column kH1 + c),
          // c < 2k.  Lanes 0..15 hold the rows (M = 64 layout, rows 16 q ..
          // 16 q + 15).  Lanes 0..15 convert column c, lanes 16..31 column
          // c + kH1/2 of the same rows (by shuffle); then even lanes store the
          // bf16 pair of rows (rr, rr + 1), which are adjacent in the K-major
          // operand.  Rows 2k .. kH1 - 1 of the operand hold zeros or values
          // of an earlier segment: they only reach G columns that are not
          // drained.
          constexpr int kLaneCols = kH1 / 2;
          const bool upper = lane >= 16;
          const int rr = 16 * q + (lane & 15);
          // in phases over all columns, so that the shuffles of different
          // columns are in flight together
          float w[kLaneCols];
          uint32_t hs[kLaneCols], ls[kLaneCols];
#pragma unroll
          for (int c0 = 0; c0 < kLaneCols; ++c0) w[c0] = d1[c0 + kLaneCols] + d1[kH1 + c0 + kLaneCols];
#pragma unroll
          for (int c0 = 0; c0 < kLaneCols; ++c0) w[c0] = __shfl_sync(0xffffffffu, w[c0], lane & 15);
          float xs[kLaneCols];
#pragma unroll
          for (int c0 = 0; c0 < kLaneCols; ++c0) {
            float x = upper ? w[c0] : d1[c0] + d1[kH1 + c0];
            // FP32 data: the data row's W = hi-row product + lo-row product
            // (adjacent rows sit in adjacent lanes; a + b == b + a, so both
            // lanes hold the same value)
            if (sv.pair_sum) x += __shfl_xor_sync(0xffffffffu, x, 1);
            xs[c0] = x;
          }
          if constexpr (kHalves) {
            // W of the view = this half's product + the other half's: send
            // ours into the other half's buffer b (once it has read the one
            // of tile jg - 2), take theirs from ours; both CTAs add the same
            // two numbers (a + b == b + a), so they hold the same W
            // Row rr of a buffer holds the lanes' column halves at floats
            // 0 .. 11 and 12 .. 23 (three 16-byte stores each, padded with
            // zeros when kH1 = 20).  The stores of a warp are released by one
            // arrival from lane 0 after the warp's barrier, so a barrier
            // phase counts the four epilogue warps.
            static_assert(2 * ((kLaneCols + 3) / 4 * 4) <= L::kXC && kLaneCols <= 12, "exchange row");
            const int xo = rr * L::kXC + (upper ? 12 : 0);
            // (the waits' verdicts are made warp-uniform: the shuffles below
            // need every lane)
            if (jg >= 2 &&
                !(ok = __all_sync(0xffffffffu, mbar_wait_cluster(bar(kXFree + b), ((jg - 2) >> 1) & 1, abort_flag, wl))))
              break;
            {
              float v[12];
#pragma unroll
              for (int c0 = 0; c0 < 12; ++c0) v[c0] = c0 < kLaneCols ? xs[c0 < kLaneCols ? c0 : 0] : 0.f;
              const uint32_t rx = map_peer(smem_u32(xbuf + b * kRows * L::kXC + xo), hpeer);
#pragma unroll
              for (int u = 0; u < 3; ++u) st_cluster_v4(rx + 16 * u, v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(map_peer(bar(kXFull + b), hpeer));
            if (!(ok = __all_sync(0xffffffffu, mbar_wait_cluster(bar(kXFull + b), (jg >> 1) & 1, abort_flag, wl))))
              break;
            {
              const float4* mine = reinterpret_cast<const float4*>(xbuf + b * kRows * L::kXC + xo);
              float v[12];
#pragma unroll
              for (int u = 0; u < 3; ++u) {
                const float4 t = mine[u];
                v[4 * u] = t.x;
                v[4 * u + 1] = t.y;
                v[4 * u + 2] = t.z;
                v[4 * u + 3] = t.w;
              }
#pragma unroll
              for (int c0 = 0; c0 < kLaneCols; ++c0) xs[c0] += v[c0];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(map_peer(bar(kXFree + b), hpeer));
          }
#pragma unroll
          for (int c0 = 0; c0 < kLaneCols; ++c0) {
            const __nv_bfloat16 hi = __float2bfloat16_rn(xs[c0]);
            const __nv_bfloat16 lo = __float2bfloat16_rn(xs[c0] - __bfloat162float(hi));
            hs[c0] = __bfloat16_as_ushort(hi);
            ls[c0] = __bfloat16_as_ushort(lo);
          }
#pragma unroll
          for (int c0 = 0; c0 < kLaneCols; ++c0) {
            hs[c0] |= __shfl_down_sync(0xffffffffu, hs[c0], 1) << 16;
            ls[c0] |= __shfl_down_sync(0xffffffffu, ls[c0], 1) << 16;
          }
          if ((lane & 1) == 0) {
#pragma unroll
            for (int c0 = 0; c0 < kLaneCols; ++c0) {
              const int c = upper ? c0 + kLaneCols : c0;
              if (c < sv.k2) {
                const uint32_t off = swz(view * L::kHalf + c, rr);
                *reinterpret_cast<uint32_t*>(wb + off) = hs[c0];
                *reinterpret_cast<uint32_t*>(wb + L::kWs + off) = ls[c0];
              }
            }
          }
        }
        fence_proxy_async();
        mbar_arrive(bar(esync));
        if (threadIdx.x == lead) {
          // all rows written: push this view's rows (hi and lo) into the peer's
          // buffer b (two views), then release our own GEMM 2 (the group's
          // barrier completes once per tile of the group)
          if (!(ok = mbar_wait(bar(esync), (jg >> 1) & 1, abort_flag, wl))) break;
          if constexpr (!kSolo) {
            const uint32_t pbar = map_peer(bar(kWPeer + b), peer);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const uint32_t src = smem_u32(wb + h * L::kWs + view * L::kWHalf);
              bulk_to_peer(map_peer(src, peer), src, L::kWHalf, pbar);
            }
          }
          mbar_arrive(bar(kWReady + b));
        }
      }
      if (!ok) break;
      // this segment's G (group 0): drain to its partial slab, then free the
      // accumulators for the next segment's GEMM 2
      if (grp == 0) {
      if (!(ok = mbar_wait(bar(kGDone), sp & 1, abort_flag, wl))) break;
      tc_fence_after();
      {
        // the slab is column-major (D rows, kNvs k2 columns): the 32 lanes
        // of a warp hold 32 consecutive rows, so every store of a column is
        // one 128-byte line
        const int D = sv.d0 + sv.d1;
        const int dv = view == 0 ? sv.d0 : sv.d1;
        for (int p = 0; p < npairs; ++p) {
          float g[L::kN2];
#pragma unroll
          for (int c = 0; c < L::kN2; c += 16) tmem_ld16(tmem + lane_off + (uint32_t)(kTG + p * L::kN2 + c), &g[c]);
          tmem_ld_wait();
          const int col = 128 * (sv.pb + p) + rg;
          if (col < dv) {
            float* o = sv.out + view * sv.d0 + col;
#pragma unroll
            for (int c = 0; c < (kSolo ? L::kHalf : L::kNW); ++c) {
              const int vv = c / L::kHalf, cc = c - vv * L::kHalf;
              if (cc < sv.k2) o[(int64_t)(vv * sv.k2 + cc) * D] = g[c] + g[L::kNW + c];  // hi + lo products
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(bar(kGFree));
      }
      ++sp;
    }
    if (ok) {
      // the peer's last end-of-GEMM-2 signal of this group's buffer (tile
      // jg - 2 or jg - 1, not waited in the loop) must have reached us
      // before we leave
      for (int j = max(0, jg - 2); j < jg; ++j)
        if ((j & 1) == grp) mbar_wait(bar(kWFree + (j & 1)), (j >> 1) & 1, abort_flag);
    }
    tc_fence_before();
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicExch(a.err, kFlagTimeout);
  cluster_sync();  // no bulk copy or remote arrive targets a CTA that has left
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Phi image: per view, K-boxes of 64 columns; B rows 0..23 hold the bf16 hi
// parts of the 2k columns [U | eta], rows 24..47 their lo parts (x - hi);
// 128B-swizzled.  Phi is then rounded in place to hi + lo so that the point
// the pass evaluates is exactly the point the solver holds.  One thread per
// element of Phi (both views in one launch); the padding of the image is
// zero from its allocation and never written.
// Columns col0 .. col0 + ng - 1 of Phi (row stride k2) form the image (a
// column group: plans with 2k > 24 run the pass once per group).
__global__ void phi_image_kernel(double* __restrict__ Phix, double* __restrict__ Phiy, int dx, int dy, int k2,
                                 int col0, int ng, int h1, uint8_t* __restrict__ img, int64_t img_view,
                                 const int* done) {
  if (done != nullptr && *done) return;
  const int v = blockIdx.y;
  const int d = v == 0 ? dx : dy;
  double* Phi = v == 0 ? Phix : Phiy;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;  // (data column j, group column c)
  if (e >= d * ng) return;
  const int j = e / ng, c = e - j * ng;
  double* px = Phi + (int64_t)j * k2 + col0 + c;
  const double x = *px;
  const __nv_bfloat16 hi = __double2bfloat16(x);
  const __nv_bfloat16 lo = __double2bfloat16(x - (double)__bfloat162float(hi));
  uint8_t* base = img + (int64_t)v * img_view + (int64_t)(j >> 6) * (2 * h1 * 128);
  *reinterpret_cast<__nv_bfloat16*>(base + swz(c, j & 63)) = hi;
  *reinterpret_cast<__nv_bfloat16*>(base + swz(h1 + c, j & 63)) = lo;
  *px = (double)__bfloat162float(hi) + (double)__bfloat162float(lo);
}

// G (D x 4k, FP64) = sum over clusters of the FP32 partials, in cluster
// order.  A CTA covers 256 consecutive entries: 64 float4 groups x 4 quarters
// of the partials; each quarter is summed with Neumaier-compensated FP32
// arithmetic (8 loads in flight), then the four (sum, compensation) pairs are
// combined in fixed order.  Error ~2 ulp of the sum, far below the partials'
// own rounding.
// `stride` is the distance of the partial slabs (floats, a multiple of 4, at
// least len); entries len .. stride - 1 of a slab are padding.  A slab is
// column-major with D = len / (nvs ng) rows: its columns are, for CCA
// (nvs = 2), the view-x then the view-y products of group columns 0 .. ng - 1
// (one view: nvs = 1), and entry (row, vv ng + c) goes to G column
// vv k2 + col0 + c of the row-major G (rows of nvs k2).  A plan with one
// column group passes ng = k2, col0 = 0.
// Gt (optional) receives the same values column-major (nvs k2 rows of D):
// the slabs' order, so these stores are coalesced and the Gram kernel reads
// them so.
__global__ void __launch_bounds__(256) tc_reduce_kernel(const float* __restrict__ part, int nparts, int64_t len,
                                                        int64_t stride, double* __restrict__ G, const int* done,
                                                        const int* nparts_dev, int ng, int col0, int k2, int nvs,
                                                        double* __restrict__ Gt) {
  if (done != nullptr && *done) return;
  if (nparts_dev != nullptr) nparts = *nparts_dev;  // batched pass: the schedule's slab count
  __shared__ float4 red_s[4][64], red_c[4][64];
  const int g = threadIdx.x & 63, qtr = threadIdx.x >> 6;
  const int64_t e4 = (int64_t)blockIdx.x * 64 + g;  // float4 group
  const bool in = 4 * e4 < len;
  const int per = (nparts + 3) / 4;
  const int p0 = qtr * per, p1 = min(nparts, p0 + per);
  float s[4] = {0.f, 0.f, 0.f, 0.f}, cp[4] = {0.f, 0.f, 0.f, 0.f};
  if (in) {
    const float4* src = reinterpret_cast<const float4*>(part) + e4;
    const int64_t stride4 = stride / 4;
    for (int b0 = p0; b0 < p1; b0 += 8) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (b0 + u < p1) ? src[(int64_t)(b0 + u) * stride4] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float x[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float t = s[i] + x[i];
          cp[i] += (fabsf(s[i]) >= fabsf(x[i])) ? ((s[i] - t) + x[i]) : ((x[i] - t) + s[i]);
          s[i] = t;
        }
      }
    }
  }
  red_s[qtr][g] = make_float4(s[0], s[1], s[2], s[3]);
  red_c[qtr][g] = make_float4(cp[0], cp[1], cp[2], cp[3]);
  __syncthreads();
  if (qtr == 0 && in) {
    double out[4];
    for (int i = 0; i < 4; ++i) out[i] = 0.0;
    for (int q = 0; q < 4; ++q) {
      const float4 a = red_s[q][g], c = red_c[q][g];
      out[0] += (double)a.x + (double)c.x;
      out[1] += (double)a.y + (double)c.y;
      out[2] += (double)a.z + (double)c.z;
      out[3] += (double)a.w + (double)c.w;
    }
    const int64_t D = len / (nvs * ng);
    for (int i = 0; i < 4; ++i) {
      const int64_t idx = 4 * e4 + i;
      if (idx >= len) continue;
      const int col = (int)(idx / D);
      const int64_t row = idx - (int64_t)col * D;
      const int vv = col / ng, c = col - vv * ng;
      G[row * nvs * k2 + vv * k2 + col0 + c] = out[i];
      if (Gt != nullptr) Gt[(int64_t)(vv * k2 + col0 + c) * D + row] = out[i];
    }
  }
}

// W^T W = Phi_bd^T G (4k x 4k), Phi_bd = blkdiag(Phi_x, Phi_y), in FP64: one
// warp per entry, lanes over rows, fixed shuffle tree, G read column-major
// (Gt: NC rows of D = dx + dy).  One view (nv = 1, FDA): Phi^T G (2k x 2k).
__global__ void tc_gram_kernel(const double* __restrict__ Phix, const double* __restrict__ Phiy, int dx, int dy,
                               int k2, int nv, const double* __restrict__ Gt, double* __restrict__ Gram,
                               const int* done) {
  if (done != nullptr && *done) return;
  const int k4 = nv * k2;
  const int e = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (e >= k4 * k4) return;
  const int a = e / k4, b = e - a * k4;
  const int v = a < k2 ? 0 : 1;
  const int ca = a - v * k2;
  const double* Phi = v == 0 ? Phix : Phiy;
  const int d = v == 0 ? dx : dy;
  const int off = v == 0 ? 0 : dx;
  double s = 0;
  const double* gb = Gt + (int64_t)b * (dx + dy) + off;
  for (int j = lane; j < d; j += 32) s += Phi[(int64_t)j * k2 + ca] * gb[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) Gram[e] = s;
}

}  // namespace tc

// ----------------------------------------------------------------- host side
namespace {

int make_map(CUtensorMap* map, const void* base, int64_t n, int d, int64_t ld) {
  return make_tma_map_bf16(map, base, n, d, ld, tc::kRows);
}

}  // namespace

// The tensor-core pass serves CCA plans with BF16 data (or FP32 data through
// the interleaved copy), dx, dy <= 1024 (views wider than 512 columns in
// 4-CTA clusters, each view's column pairs split over two CTAs), 16-byte
// aligned rows (ld a multiple of 8) and 16-byte aligned bases; Phi columns
// beyond 24 per view (k > 12, up to the library's k <= 20) are taken in a
// second column group, which reads the data a second time.  FDA plans with
// FP32 data and d <= 1024 stream the interleaved copy of their class-centred
// rows in one-view clusters (the view's column pairs split over two CTAs).
bool tc_pass_eligible(const Plan& p) {
  if (p.kind == kLDA) return p.dtype == GBCCA_FP32 && 2 * p.k <= 2 * tc::kHalfMax && p.v[0].d <= 1024 && p.ts_ready;
  if (p.kind != kCCA || 2 * p.k > 2 * tc::kHalfMax || p.v[0].d > 1024 || p.v[1].d > 1024) return false;
  if (p.dtype == GBCCA_FP32) return p.ts_ready;  // the plan's own aligned copy
  if (p.dtype != GBCCA_BF16) return false;
  for (int v = 0; v < 2; ++v) {
    if (p.v[v].ld % 8 != 0 || (reinterpret_cast<uintptr_t>(p.v[v].Z) & 15) != 0) return false;
  }
  return true;
}

// Column groups of Phi for the tensor-core pass: one group for 2k <= 24,
// else two of ng0 = k rounded up to even columns (an even group keeps every
// partial slab a multiple of 4 floats), each at most 24.
int tc_groups(const Plan& p) { return 2 * p.k <= tc::kHalfMax ? 1 : 2; }
static void tc_group(const Plan& p, int g, int* col0, int* ng) {
  const int k2 = 2 * p.k;
  if (tc_groups(p) == 1) {
    *col0 = 0;
    *ng = k2;
    return;
  }
  const int ng0 = (p.k + 1) / 2 * 2;
  *col0 = g * ng0;
  *ng = g == 0 ? ng0 : k2 - ng0;
}
// one-view plans (FDA): clusters of two CTAs that split the view's column
// pairs
static bool tc_solo(const Plan& p) { return p.kind == kLDA; }
static int tc_group_h1(const Plan& p, int ng) { return ng <= 20 ? 20 : tc::kHalfMax; }
// views wider than 512 columns: 4-CTA clusters and images of 16 K-boxes
bool tc_quad(const Plan& p) { return p.kind == kCCA && std::max(p.v[0].d, p.v[1].d) > 512; }
// bytes between the views' images of a group (one-view plans: 16 K-boxes,
// the second CTA's pairs starting at K-box 8 at most)
static int64_t tc_img_view(const Plan& p) { return (tc_quad(p) || tc_solo(p) ? 2 : 1) * (int64_t)tc::kPhiView; }
static int tc_nviews(const Plan& p) { return tc_solo(p) ? 1 : 2; }
static uint8_t* tc_group_img(const Plan& p, int g) { return p.tc_img + (int64_t)g * tc_nviews(p) * tc_img_view(p); }
// floats of one cluster's partial slab of a group of ng columns: D x 2 ng
// (one view: d x ng, rounded up to a multiple of 4)
static int64_t tc_slab(const Plan& p, int ng) { return ((int64_t)p.D * tc_nviews(p) * ng + 3) / 4 * 4; }
// partial slabs of group g: clusters (at most half the SMs) x one slab each
static float* tc_group_part(const Plan& p, int g) {
  int col0 = 0, ng0 = 0;
  tc_group(p, 0, &col0, &ng0);
  return p.tc_part + (int64_t)g * (p.sm_count / 2) * tc_slab(p, ng0);
}

// The Phi images of a plan (both views, every column group), group g with
// h1 rows per half (h1 = 0: each group's own); also rounds Phi to the bf16
// hi + lo point the pass evaluates.
int tc_phi_image(Plan& p, int h1, cudaStream_t st, const int* done) {
  const int k2 = 2 * p.k;
  const int nv = tc_nviews(p);
  const int d1 = nv > 1 ? p.v[1].d : 0;
  double* Phi1 = nv > 1 ? p.v[1].Phi : p.v[0].Phi;
  const int dmax = std::max(p.v[0].d, d1);
  for (int g = 0; g < tc_groups(p); ++g) {
    int col0 = 0, ng = 0;
    tc_group(p, g, &col0, &ng);
    const int hg = h1 > 0 ? h1 : tc_group_h1(p, ng);
    tc::phi_image_kernel<<<dim3(ceil_div(dmax * ng, 256), nv), 256, 0, st>>>(
        p.v[0].Phi, Phi1, p.v[0].d, d1, k2, col0, ng, hg, tc_group_img(p, g), tc_img_view(p), done);
    GB_CHECK_LAUNCH();
  }
  return GBCCA_OK;
}

// The streamed matrices of an eligible plan: the caller's BF16 matrices, or
// for FP32 data the plan's row-interleaved hi/lo copy (2n rows).  One-view
// plans stream view 0 (the second entry repeats it and is not read).
static void tc_sources(const Plan& p, const void* src[2], int64_t ld[2], int64_t* rows) {
  const bool fp32 = p.dtype == GBCCA_FP32;
  *rows = fp32 ? 2 * p.n : p.n;
  for (int v = 0; v < 2; ++v) {
    const int u = v < tc_nviews(p) ? v : 0;
    src[v] = fp32 ? (const void*)p.ts_copy[u] : p.v[u].Z;
    ld[v] = fp32 ? p.ts_ld[u] : p.v[u].ld;
  }
}

int tc_pass(Plan& p, cudaStream_t st, const int* done) {
  // FP32 data: the row-interleaved hi/lo copy (2n rows) made when the data
  // was bound; BF16 data: the caller's matrices
  const bool fp32 = p.dtype == GBCCA_FP32;
  int64_t rows = 0;
  const void* src[2];
  int64_t ld[2];
  tc_sources(p, src, ld, &rows);
  const bool solo = tc_solo(p);
  const int nv = tc_nviews(p);
  if (p.tc_map_for[0] != src[0] || p.tc_map_for[1] != src[1]) {
    for (int v = 0; v < 2; ++v)
      GB_TRY(make_map(reinterpret_cast<CUtensorMap*>(p.tc_map[v]), src[v], rows, p.v[v < nv ? v : 0].d, ld[v]));
    p.tc_map_for[0] = src[0];
    p.tc_map_for[1] = src[1];
  }
  const int k2 = 2 * p.k, k4 = nv * k2;
  GB_TRY(tc_phi_image(p, 0, st, done));
  const CUtensorMap* mx = reinterpret_cast<const CUtensorMap*>(p.tc_map[0]);
  const CUtensorMap* my = reinterpret_cast<const CUtensorMap*>(p.tc_map[1]);
  const int groups = tc_groups(p);
  if (p.kev0 != nullptr) GB_CUDA(record_timing_event(p.kev0, st));
  int ncl = 1;
  for (int g = 0; g < groups; ++g) {
    int col0 = 0, ng = 0;
    tc_group(p, g, &col0, &ng);
    const int h1 = tc_group_h1(p, ng);  // Phi image rows per half (GEMM 1 N = 2 h1)
    tc::Args a{};
    a.n = p.n;
    for (int v = 0; v < 2; ++v) {
      a.d[v] = v < nv ? p.v[v].d : 0;
      a.pairs[v] = ceil_div(a.d[v], 128);
    }
    a.k2 = ng;
    a.slab = tc_slab(p, ng);
    a.wait_limit = p.opt.wait_cycles > 0 ? p.opt.wait_cycles : tc::kWaitCycles;
    a.ntiles = ceil_div(rows, tc::kRows);
    a.pair_sum = fp32 ? 1 : 0;
    a.phi_img = tc_group_img(p, g);
    a.img_view = tc_img_view(p);
    a.partG = tc_group_part(p, g);
    a.err = p.flag;
    a.done = done;
    const bool quad = tc_quad(p);
    const int csz = quad ? 4 : 2;  // CTAs per cluster
    auto kern = solo ? (h1 == 20 ? tc::tc_pass_kernel<20, false, true> : tc::tc_pass_kernel<tc::kHalfMax, false, true>)
                : quad ? (h1 == 20 ? tc::tc_pass_kernel<20, true> : tc::tc_pass_kernel<tc::kHalfMax, true>)
                       : (h1 == 20 ? tc::tc_pass_kernel<20> : tc::tc_pass_kernel<tc::kHalfMax>);
    const int smem = solo ? (h1 == 20 ? tc::Lay<20, false, true>::kSmemBytes : tc::Lay<tc::kHalfMax, false, true>::kSmemBytes)
                     : quad ? (h1 == 20 ? tc::Lay<20, true>::kSmemBytes : tc::Lay<tc::kHalfMax, true>::kSmemBytes)
                            : (h1 == 20 ? tc::Lay<20>::kSmemBytes : tc::Lay<tc::kHalfMax>::kSmemBytes);
    GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csz;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(tc::kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (p.tc_clusters <= 0) {
      // persistent grid: as many clusters as can be resident at once
      cfg.gridDim = dim3(csz * (p.sm_count / csz), 1, 1);
      int nc = 0;
      GB_CUDA(cudaOccupancyMaxActiveClusters(&nc, kern, &cfg));
      p.tc_clusters = std::max(1, std::min(nc, p.sm_count / csz));
    }
    ncl = std::min(p.tc_clusters, a.ntiles);
    cfg.gridDim = dim3(csz * ncl, 1, 1);
    GB_CUDA(cudaLaunchKernelEx(&cfg, kern, *mx, *my, a));
    GB_CHECK_LAUNCH();
  }
  if (p.kev1 != nullptr) GB_CUDA(record_timing_event(p.kev1, st));
  if (p.fork_after_pass) {
    // work that needs only Phi may start beside the reduction
    GB_CUDA(cudaEventRecord(p.pass_fork, st));
    p.pass_forked = true;
  }
  for (int g = 0; g < groups; ++g) {
    int col0 = 0, ng = 0;
    tc_group(p, g, &col0, &ng);
    // partial slabs, one per cluster
    const int64_t len = (int64_t)p.D * nv * ng;
    tc::tc_reduce_kernel<<<ceil_div(len, 256), 256, 0, st>>>(tc_group_part(p, g), ncl, len, tc_slab(p, ng), p.G,
                                                             done, nullptr, ng, col0, k2, nv, p.Gt);
    GB_CHECK_LAUNCH();
  }
  tc::tc_gram_kernel<<<ceil_div(k4 * k4 * 32, 256), 256, 0, st>>>(
      p.v[0].Phi, nv > 1 ? p.v[1].Phi : p.v[0].Phi, p.v[0].d, nv > 1 ? p.v[1].d : 0, k2, nv, p.Gt, p.Gram, done);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}


// ------------------------------------------------------------ batched pass
// Several plans' passes in one persistent launch (same kernel, segment
// schedule).  The instance table, the segments and the per-instance slab
// counts live in device memory, so a captured graph keeps one launch while
// the schedule is rewritten between replays (finished plans drop out).
struct TcBatch {
  bool quad = false;           // 4-CTA clusters (plans with a view wider than 512)
  int csz = 2;                 // CTAs per cluster
  int n = 0;                   // table entries: one per (plan, column group)
  int nplans = 0;
  int h1 = tc::kHalfMax;       // Phi image rows per half, common to the batch
  std::vector<int64_t> rows;   // streamed rows per entry
  std::vector<int> first;      // per plan: its first entry (entries first .. first + count - 1)
  std::vector<int> count;
  std::vector<int64_t> plan_bytes;  // algorithmic bytes of one pass per plan
  tc::Inst* inst_h = nullptr;  // pinned host copies of the tables
  tc::Seg* seg_h = nullptr;
  int* off_h = nullptr;
  int* nparts_h = nullptr;
  tc::Inst* inst_d = nullptr;
  tc::Seg* seg_d = nullptr;
  int* off_d = nullptr;
  int* nparts_d = nullptr;
  int* err_d = nullptr;
  int max_clusters = 0;        // clusters the tables have room for
  int clusters = 0;            // clusters of the current schedule
  int max_segs = 0;
};

void tc_batch_destroy(TcBatch* b) {
  if (b == nullptr) return;
  cudaFreeHost(b->inst_h);
  cudaFreeHost(b->seg_h);
  cudaFreeHost(b->off_h);
  cudaFreeHost(b->nparts_h);
  cudaFree(b->inst_d);
  cudaFree(b->seg_d);
  cudaFree(b->off_d);
  cudaFree(b->nparts_d);
  cudaFree(b->err_d);
  delete b;
}

// Instance table of the plans (each eligible for the tensor-core pass, with
// its data bound); copied to the device on `st`.
TcBatch* tc_batch_create(Plan* const* plans, int n, cudaStream_t st, int* rc) {
  *rc = GBCCA_OK;
  auto* b = new (std::nothrow) TcBatch();
  if (b == nullptr) {
    *rc = GBCCA_ERR_OOM;
    return nullptr;
  }
  b->nplans = n;
  b->quad = n > 0 && tc_quad(*plans[0]);
  b->csz = b->quad ? 4 : 2;
  int entries = 0, h1 = 20, sm = 1;
  for (int i = 0; i < n; ++i) {
    b->first.push_back(entries);
    b->count.push_back(tc_groups(*plans[i]));
    for (int g = 0; g < tc_groups(*plans[i]); ++g) {
      int col0 = 0, ng = 0;
      tc_group(*plans[i], g, &col0, &ng);
      h1 = std::max(h1, tc_group_h1(*plans[i], ng));
    }
    entries += tc_groups(*plans[i]);
    sm = std::max(sm, plans[i]->sm_count);
  }
  b->n = entries;
  b->h1 = h1;
  b->max_clusters = std::max(1, sm / b->csz);
  b->max_segs = b->max_clusters + entries + 1;  // a contiguous partition has at most clusters + entries pieces
  const int n1 = std::max(entries, 1);
  bool ok = cudaMallocHost(&b->inst_h, sizeof(tc::Inst) * n1) == cudaSuccess &&
            cudaMallocHost(&b->seg_h, sizeof(tc::Seg) * b->max_segs) == cudaSuccess &&
            cudaMallocHost(&b->off_h, sizeof(int) * (b->max_clusters + 1)) == cudaSuccess &&
            cudaMallocHost(&b->nparts_h, sizeof(int) * n1) == cudaSuccess &&
            cudaMalloc(&b->inst_d, sizeof(tc::Inst) * n1) == cudaSuccess &&
            cudaMalloc(&b->seg_d, sizeof(tc::Seg) * b->max_segs) == cudaSuccess &&
            cudaMalloc(&b->off_d, sizeof(int) * (b->max_clusters + 1)) == cudaSuccess &&
            cudaMalloc(&b->nparts_d, sizeof(int) * n1) == cudaSuccess &&
            cudaMalloc(&b->err_d, sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    tc_batch_destroy(b);
    set_last_error("allocation of the batch schedule failed");
    *rc = GBCCA_ERR_OOM;
    return nullptr;
  }
  std::memset(b->inst_h, 0, sizeof(tc::Inst) * n1);
  b->rows.assign(entries, 0);
  b->plan_bytes.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    Plan& p = *plans[i];
    const void* src[2];
    int64_t ld[2], rows = 0;
    tc_sources(p, src, ld, &rows);
    b->plan_bytes[i] = rows * (int64_t)(p.v[0].d + p.v[1].d) * 2;
    for (int g = 0; g < b->count[i]; ++g) {
      const int e = b->first[i] + g;
      tc::Inst& I = b->inst_h[e];
      b->rows[e] = rows;
      for (int v = 0; v < 2; ++v) {
        *rc = make_map(&I.map[v], src[v], rows, p.v[v].d, ld[v]);
        if (*rc != GBCCA_OK) {
          tc_batch_destroy(b);
          return nullptr;
        }
        I.d[v] = p.v[v].d;
        I.pairs[v] = ceil_div(p.v[v].d, 128);
      }
      int col0 = 0, ng = 0;
      tc_group(p, g, &col0, &ng);
      I.phi_img = tc_group_img(p, g);
      I.img_view = tc_img_view(p);
      I.partG = tc_group_part(p, g);
      I.done = &p.st->done;
      I.k2 = ng;
      I.pair_sum = p.dtype == GBCCA_FP32 ? 1 : 0;
      I.slab = (int64_t)p.D * 2 * ng;
    }
  }
  cudaError_t e = cudaMemcpyAsync(b->inst_d, b->inst_h, sizeof(tc::Inst) * n1, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->err_d, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_error(std::string("batch table upload: ") + cudaGetErrorString(e));
    tc_batch_destroy(b);
    *rc = GBCCA_ERR_CUDA;
    return nullptr;
  }
  return b;
}

int tc_batch_h1(const TcBatch* b) { return b->h1; }
int* tc_batch_err(TcBatch* b) { return b->err_d; }
int tc_batch_max_clusters(const TcBatch* b) { return b->max_clusters; }
int tc_batch_clusters(const TcBatch* b) { return b->clusters; }
// Algorithmic bytes of one batched pass over the active plans (each plan's
// data once, whatever its column groups).
int64_t tc_batch_bytes(const TcBatch* b, const bool* active) {
  int64_t s = 0;
  for (int i = 0; i < b->nplans; ++i)
    if (active == nullptr || active[i]) s += b->plan_bytes[i];
  return s;
}

// Schedule of the active instances over `clusters` 2-CTA clusters: their
// 64-row tiles, each weighted by 2 + the pairs of its wider view (the two
// CTAs of a cluster move through a tile together, and a tile costs a fixed
// epilogue and exchange on top of its MMAs), are cut into `clusters`
// contiguous ranges of near-equal weight.  The pieces of instance i (one per
// cluster it reaches) write its slabs 0, 1, ... in order, and its reduction
// adds that many slabs.  The tables go
// to the device on `st`; the pinned host copies are rewritten only by the
// next schedule, after the caller has synchronized `st`.
int tc_batch_schedule(TcBatch* b, const bool* plan_active, int clusters, cudaStream_t st) {
  clusters = std::max(1, std::min(clusters, b->max_clusters));
  std::vector<char> active(b->n, 0);  // per entry
  for (int i = 0; i < b->nplans; ++i)
    for (int g = 0; g < b->count[i]; ++g) active[b->first[i] + g] = plan_active[i] ? 1 : 0;
  // pairs of a tile per CTA (4-CTA clusters: each view's pairs over two CTAs)
  auto cta_pairs = [&](int i) {
    const int P = std::max(b->inst_h[i].pairs[0], b->inst_h[i].pairs[1]);
    return b->quad ? (P + 1) / 2 : P;
  };
  int64_t total = 0;
  for (int i = 0; i < b->n; ++i) {
    b->nparts_h[i] = 0;
    if (active[i]) total += ceil_div(b->rows[i], (int64_t)tc::kRows) * (2 + cta_pairs(i));
  }
  int c = 0, nseg = 0;
  int64_t cum = 0;
  b->off_h[0] = 0;
  auto bound = [&](int cc) { return (total * (cc + 1) + clusters - 1) / clusters; };
  for (int i = 0; i < b->n; ++i) {
    if (!active[i]) continue;
    const int64_t tiles = ceil_div(b->rows[i], (int64_t)tc::kRows);
    const int64_t w = 2 + cta_pairs(i);
    int pieces = 0;  // segments of instance i so far = its next slab
    int64_t t = 0;
    while (t < tiles) {
      int64_t take = tiles - t;
      if (c < clusters - 1) take = std::min(take, (bound(c) - cum) / w);
      if (take <= 0) {  // this cluster is full: close it
        b->off_h[++c] = nseg;
        continue;
      }
      b->seg_h[nseg++] = tc::Seg{i, (int)t, (int)take, pieces++};
      t += take;
      cum += take * w;
      if (c < clusters - 1 && cum >= bound(c)) b->off_h[++c] = nseg;
    }
    b->nparts_h[i] = pieces;
  }
  while (c < clusters) b->off_h[++c] = nseg;
  b->clusters = clusters;
  GB_CUDA(cudaMemcpyAsync(b->seg_d, b->seg_h, sizeof(tc::Seg) * std::max(nseg, 1), cudaMemcpyHostToDevice, st));
  GB_CUDA(cudaMemcpyAsync(b->off_d, b->off_h, sizeof(int) * (clusters + 1), cudaMemcpyHostToDevice, st));
  GB_CUDA(cudaMemcpyAsync(b->nparts_d, b->nparts_h, sizeof(int) * std::max(b->n, 1), cudaMemcpyHostToDevice, st));
  return GBCCA_OK;
}

// The Phi images of a batch member (h1 of the batch); nothing once the plan
// has finished.
int tc_batch_pre(const TcBatch* b, Plan& p, cudaStream_t st) { return tc_phi_image(p, b->h1, st, &p.st->done); }

// One launch over every scheduled tile of the batch.
int tc_batch_launch(TcBatch* b, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  tc::Args a{};
  a.err = b->err_d;
  a.insts = b->inst_d;
  a.segs = b->seg_d;
  a.seg_off = b->off_d;
  auto kern = b->quad ? (b->h1 == 20 ? tc::tc_pass_kernel<20, true> : tc::tc_pass_kernel<tc::kHalfMax, true>)
                      : (b->h1 == 20 ? tc::tc_pass_kernel<20> : tc::tc_pass_kernel<tc::kHalfMax>);
  const int smem = b->quad ? (b->h1 == 20 ? tc::Lay<20, true>::kSmemBytes : tc::Lay<tc::kHalfMax, true>::kSmemBytes)
                           : (b->h1 == 20 ? tc::Lay<20>::kSmemBytes : tc::Lay<tc::kHalfMax>::kSmemBytes);
  GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = b->csz;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(tc::kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(b->csz * std::max(1, b->clusters), 1, 1);
  // the tensor-map parameters are unused in batch mode; any valid map will do
  const CUtensorMap* m0 = &b->inst_h[0].map[0];
  const CUtensorMap* m1 = &b->inst_h[0].map[1];
  if (e0 != nullptr) GB_CUDA(record_timing_event(e0, st));
  GB_CUDA(cudaLaunchKernelEx(&cfg, kern, *m0, *m1, a));
  GB_CHECK_LAUNCH();
  if (e1 != nullptr) GB_CUDA(record_timing_event(e1, st));
  return GBCCA_OK;
}

// Sum of plan i's slabs (every column group) into its G, then its Gram.
int tc_batch_post(const TcBatch* b, int i, Plan& p, cudaStream_t st, const int* done) {
  const int k2 = 2 * p.k, k4 = 4 * p.k;
  const int groups = b->count[i];
  for (int g = 0; g < groups; ++g) {
    int col0 = 0, ng = 0;
    tc_group(p, g, &col0, &ng);
    const int64_t len = (int64_t)p.D * 2 * ng;
    tc::tc_reduce_kernel<<<ceil_div(len, 256), 256, 0, st>>>(tc_group_part(p, g), 1, len, len, p.G, done,
                                                             b->nparts_d + b->first[i] + g, ng, col0, k2, 2, p.Gt);
    GB_CHECK_LAUNCH();
  }
  tc::tc_gram_kernel<<<ceil_div(k4 * k4 * 32, 256), 256, 0, st>>>(p.v[0].Phi, p.v[1].Phi, p.v[0].d, p.v[1].d, k2,
                                                                  2, p.Gt, p.Gram, done);
  GB_CHECK_LAUNCH();
  return GBCCA_OK;
}

}  // namespace gbcca
