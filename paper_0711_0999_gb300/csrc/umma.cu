// Tensor-core (tcgen05) path of the lattice step.
//
// Gauss-Jordan on A'_q (np x np, FP32 complex, batch of nb matrices) in
// steps of W = 128 or 256 columns.  Step k0:
//   P = inv(A_KK)   W = 128: gj_pivot_pack, in shared memory (FP32); W = 256:
//                   the 128-column Gauss-Jordan below on a copy of the
//                   256 x 256 block (gj_extract), packed by gj_ppack; P is
//                   packed bf16 hi/lo
//   gj_panel_pack   C' = A_{:,K} (C'_K = -I) packed as the update's A operand;
//                   A_{K,:}^T (A_KK -> I), 2x2 real-embedded, packed as the
//                   R-product's B operand (first step only: later steps'
//                   panels come from the update's epilogue)
//   umma_gemm       R = P A_{K,:} (bf16x3), written packed as the update's B
//   umma_gemm       A <- A (rows K, cols K zeroed) - C' R (bf16x3)
// A complex product is a real GEMM on interleaved storage: the A operand is
// the interleaved row (re, im, re, im, ...), the B operand the 2x2 real
// embedding [[re, -im], [im, re]] of each complex entry, so the output lands
// interleaved.
#include "lattice.cuh"
#include "umma.cuh"
#include "umma_core.cuh"

namespace nedmft {

using namespace umma;

namespace {

constexpr int kNb = 128;        // Gauss-Jordan block (complex columns)
constexpr int kKt = 2 * kNb / kTileK;  // K tiles of the rank-kNb products (4)

// ------------------------------------------------------------------ the GEMM kernel

// One 128 x BN output tile per CTA: C = sum over pairs of A_slice(a) B_slice(b)^T,
// K = kt * 64, accumulated in FP32 in TMEM.  Warp 0: TMA producer; warp 1:
// TMEM allocator and MMA issuer; warps 2-5: epilogue (one TMEM lane each).
struct GemmParams {
  const __nv_bfloat16* a;
  size_t a_batch;        // elements between batch entries (0: shared operand)
  size_t a_slice;        // elements between slices
  const __nv_bfloat16* b;
  size_t b_batch;
  size_t b_slice;
  int kt;                // K tiles
  int* status;
};

// The persistent kernel loads its operands in half tiles (128 rows x 32 k,
// 8 KB) through one tensor map over a buffer of packed images: 4-D, (element
// of a core-matrix row, core column of the tile, 8-row group, tile), the tile
// index counting 16 KB from the map's base.  Every operand starts at a tile
// boundary; a / b give tile indices of batch entry 0, slice 0.
struct TileMapParams {
  CUtensorMap map;
  long long a, a_batch, a_slice;  // tiles
  long long b, b_batch, b_slice;
  int kt;                          // K tiles (64 k) of the product
  int* status;
};

template <int BN, int SA, int SB, int STAGES>
struct Cfg {
  static constexpr int kBn = BN;
  static constexpr int kSa = SA;
  static constexpr int kSb = SB;
  static constexpr int kStages = STAGES;
  static constexpr int kBTiles = BN / kTileRows;
  static constexpr int kStageBytes = (SA + SB * kBTiles) * kTileBytes;
  static constexpr int kSmem = STAGES * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr uint32_t kTmemCols = BN < 32 ? 32 : BN;
};

// bf16x3: hi*hi + hi*lo + lo*hi, one accumulator.  A pair list names the
// A and B slices of each product, the accumulator it adds into (kAccs
// accumulators of kBn columns per tile) and whether it is the first product
// of that accumulator in a K step.
struct Split3 {
  static constexpr int kPairs = 3;
  static constexpr int kAccs = 1;
  __device__ static int a(int p) { return p == 2 ? 1 : 0; }
  __device__ static int b(int p) { return p == 1 ? 1 : 0; }
  __device__ static int acc(int) { return 0; }
  __device__ static bool first(int p) { return p == 0; }
};

// hi*hi alone: for a product whose own rounding lies far below the target.
struct Split1 {
  static constexpr int kPairs = 1;
  static constexpr int kAccs = 1;
  __device__ static int a(int) { return 0; }
  __device__ static int b(int) { return 0; }
  __device__ static int acc(int) { return 0; }
  __device__ static bool first(int) { return true; }
};

// Two bf16x3 products into two accumulators: A slices (hi, lo) of variant 0
// then of variant 1, one B (hi, lo); accumulator v takes A variant v times B.
// The R product uses it with A = P' = (Re P, -Im P) and P'' = (Im P, Re P)
// row-interleaved over k, and B = A_{K,:} as (Re, Im) pairs over k: the two
// accumulators are Re R and Im R.
struct Split3x2 {
  static constexpr int kPairs = 6;
  static constexpr int kAccs = 2;
  __device__ static int a(int p) { return 2 * (p / 3) + (p % 3 == 2 ? 1 : 0); }
  __device__ static int b(int p) { return p % 3 == 1 ? 1 : 0; }
  __device__ static int acc(int p) { return p / 3; }
  __device__ static bool first(int p) { return p % 3 == 0; }
};

template <class C, class Pairs, class Epi>
__device__ __forceinline__ void umma_gemm_body(const GemmParams& p, const Epi& epi) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::kStages * C::kStageBytes);
  uint64_t* empty = full + C::kStages;
  uint64_t* acc_full = empty + C::kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = blockIdx.x, mt = blockIdx.y, bidx = blockIdx.z;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, C::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      const __nv_bfloat16* a = p.a + bidx * p.a_batch;
      const __nv_bfloat16* b = p.b + bidx * p.b_batch;
      int issued = 0;
      for (int kt = 0; kt < p.kt; ++kt) {
        const int s = kt % C::kStages;
        const uint32_t ph = (kt / C::kStages) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1, abort_flag)) break;
        unsigned char* st = smem + s * C::kStageBytes;
        mbar_arrive_expect_tx(&full[s], C::kStageBytes);
        for (int sa = 0; sa < C::kSa; ++sa)
          bulk_g2s(st + sa * kTileBytes, a + sa * p.a_slice + ((size_t)mt * p.kt + kt) * kTileElems, kTileBytes,
                   &full[s]);
        for (int sb = 0; sb < C::kSb; ++sb)
          for (int u = 0; u < C::kBTiles; ++u)
            bulk_g2s(st + (C::kSa + sb * C::kBTiles + u) * kTileBytes,
                     b + sb * p.b_slice + ((size_t)(nt * C::kBTiles + u) * p.kt + kt) * kTileElems, kTileBytes,
                     &full[s]);
        issued = kt + 1;
      }
      // never leave a copy in flight: wait (bounded) for every stage issued in the last round
      for (int kt = issued - C::kStages < 0 ? 0 : issued - C::kStages; kt < issued; ++kt) {
        const int s = kt % C::kStages;
        const uint32_t ph = (kt / C::kStages) & 1;
        uint64_t t0 = global_ns();
        while (!mbar_test(&full[s], ph) && global_ns() - t0 < kDrainNs) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(128, C::kBn);
      for (int kt = 0; kt < p.kt; ++kt) {
        const int s = kt % C::kStages;
        const uint32_t ph = (kt / C::kStages) & 1;
        if (!mbar_wait(&full[s], ph, abort_flag)) break;
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * C::kStageBytes);
#pragma unroll
        for (int kk = 0; kk < kTileK / 16; ++kk) {
#pragma unroll
          for (int q = 0; q < Pairs::kPairs; ++q) {
            const uint32_t a_addr = st + Pairs::a(q) * kTileBytes + kk * 256;
            const uint32_t b_addr = st + (C::kSa + Pairs::b(q) * C::kBTiles) * kTileBytes + kk * 256;
            mma_bf16(tmem, smem_desc(a_addr, 128, 1024), smem_desc(b_addr, 128, 1024), idesc,
                     (kt > 0 || kk > 0 || q > 0) ? 1u : 0u);
          }
        }
        mma_commit(&empty[s]);
      }
      mma_commit(acc_full);
    }
  } else {
    // epilogue: warp w owns TMEM lanes 32 (w % 4) .. +31
    const int q = warp & 3;
    const int row = q * 32 + lane;
    if (mbar_wait(acc_full, 0, abort_flag)) {
      tc_fence_after();
      if (!*abort_flag) {
#pragma unroll 1
        for (int c0 = 0; c0 < C::kBn; c0 += 32) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + c0, v);
          epi(bidx, mt, nt, row, c0, v);
        }
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    // the tensor core must be idle before the columns are released
    uint64_t t0 = global_ns();
    while (!mbar_test(acc_full, 0) && global_ns() - t0 < kDrainNs) {
    }
    tc_fence_after();
    tmem_dealloc(tmem, C::kTmemCols);
  }
  if (threadIdx.x == 0 && *abort_flag && p.status) atomicCAS(p.status, 0, DS_TIMEOUT);
}

// One tile per CTA (non-persistent), skipping the matrices whose flag is 0.
template <class C, class Pairs, class Epi>
__global__ void __launch_bounds__(192, 1) umma_gemm_flag_kernel(GemmParams p, Epi epi, const int* flags, int q0) {
  if (!flags[q0 + blockIdx.z]) return;
  umma_gemm_body<C, Pairs, Epi>(p, epi);
}


using CfgGJ = Cfg<256, 2, 2, 2>;  // 128 x 256 tiles, hi/lo operands, 2 stages (192 KB)
using CfgHi = Cfg<256, 1, 1, 4>;  // 128 x 256 tiles, hi operands only, 4 stages (192 KB)

// Stages of half tiles (32 k): 4 x 48 KB for the persistent Gauss-Jordan products.
template <int BN, int SA, int SB, int STAGES>
struct CfgHalf {
  static constexpr int kBn = BN;
  static constexpr int kSa = SA;
  static constexpr int kSb = SB;
  static constexpr int kStages = STAGES;
  static constexpr int kBTiles = BN / kTileRows;
  static constexpr int kHalfBytes = kTileBytes / 2;
  static constexpr int kStageBytes = (SA + SB * kBTiles) * kHalfBytes;
  static constexpr int kBarBytes = 512;
  static constexpr int kSmem = STAGES * kStageBytes + 1024 /*align*/ + kBarBytes;
  static constexpr int kRedBuf = 2;  // staging boxes per epilogue warp
};
using CfgGJH = CfgHalf<256, 2, 2, 4>;
// The R product: 128 complex columns per tile, A slices P' and P'' (hi, lo),
// B (hi, lo) of A_{K,:}; two accumulators (Re R, Im R) of 128 columns each.
using CfgRP = CfgHalf<128, 4, 2, 4>;

// The same operands for a CTA pair, whose CTAs hold half of B each: stages of
// 32 KB instead of 48 KB.  The update (N_c = 1500) ran fastest with the freed
// shared memory spent on stages (6 stages, 2 boxes: 1.41 ms per 152-matrix
// launch; 5 and 3: 1.446; 4 and 6: 1.447; 4 and 4: 1.463).
template <class C, int STAGES, int REDBUF>
struct PairCfg : C {
  static constexpr int kStages = STAGES;
  static constexpr int kRedBuf = REDBUF;
};

// Persistent form: CTA c takes tiles c, c + G, c + 2G, ... of the linear
// order (batch, m tile, n tile), n fastest, so that at any time the CTAs work
// on about one matrix and its operand panels stay in L2.  The stage ring runs
// on across tiles and the TMEM holds two accumulators, so the epilogue of one
// tile overlaps the loads and products of the next.
//
// Epilogues with Epi::kStage stage -acc of plain tiles in shared memory, one
// 32 x 32 FP32 box (4 KB, 128-byte swizzle) per warp and column chunk, C::kRedBuf
// boxes per warp in a ring, and add it into the output at L2 with one tensor
// bulk reduction per box through Epi::red_map.  Tiles whose old values the
// epilogue needs load them into the same ring, C::kRedBuf chunks ahead.
constexpr int kRedBox = 32 * 32 * 4;
constexpr int kMaxBoxBars = 32;
template <class C, int EPIW>
constexpr int red_stage_bytes() { return 512 + EPIW * C::kRedBuf * kRedBox; }

// The barriers and flags of a persistent kernel, after its stage ring.
template <int STAGES>
struct PersistBars {
  uint64_t full[STAGES], empty[STAGES];  // stage filled / stage released by the products
  uint64_t acc_full[2], acc_empty[2];    // accumulator buffer ready / drained
  uint64_t drain;                        // every product issued by this CTA has completed
  uint64_t box[kMaxBoxBars];             // staging-box loads of the epilogue warps
  uint32_t tmem_slot;
  int abort;
};

template <class C, class Pairs, class Epi, int EPIW, int PAIR>
__global__ void __launch_bounds__(64 + 32 * EPIW, 1)
    umma_gemm_persistent_kernel(const __grid_constant__ TileMapParams p, const __grid_constant__ Epi epi, int n_tiles,
                                int m_tiles, int batch) {
  static_assert(sizeof(PersistBars<C::kStages>) <= C::kBarBytes, "barrier block");
  constexpr int kRedBuf = C::kRedBuf;
  static_assert(EPIW * kRedBuf <= kMaxBoxBars, "staging-box barriers");
  static_assert(PAIR == 1 || (PAIR == 2 && C::kBTiles == 2), "a CTA pair splits B in halves of 128 rows");
  // B half tiles per CTA and slice: a CTA of a pair holds half of B
  constexpr int kBPer = PAIR == 2 ? 1 : C::kBTiles;
  constexpr int kStageBytes = (C::kSa + C::kSb * kBPer) * C::kHalfBytes;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  auto& bars = *reinterpret_cast<PersistBars<C::kStages>*>(smem + C::kStages * kStageBytes);
  uint64_t* full = bars.full;
  uint64_t* empty = bars.empty;
  uint64_t* acc_full = bars.acc_full;
  uint64_t* acc_empty = bars.acc_empty;
  volatile int* abort_flag = &bars.abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // work units: (batch entry, m tile or pair of m tiles, n tile), n fastest
  const int per_u = n_tiles * (m_tiles / PAIR);
  const int total = per_u * batch;
  const int G = gridDim.x / PAIR;
  const int cta = blockIdx.x / PAIR;
  const int rank = PAIR == 2 ? (int)cluster_ctarank() : 0;
  constexpr uint32_t kAccCols = C::kBn * Pairs::kAccs;  // one tile's accumulators
  constexpr uint32_t kCols = 2 * kAccCols;                // two tiles in flight

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&acc_full[s], 1);
      mbar_init(&acc_empty[s], PAIR * 32 * EPIW);  // a pair: the even CTA's barrier counts both CTAs
    }
    mbar_init(&bars.drain, 1);
    if (Epi::kStage)
      for (int k = 0; k < EPIW * kRedBuf; ++k) mbar_init(&bars.box[k], 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    if constexpr (PAIR == 2) tmem_alloc_pair(&bars.tmem_slot, kCols);
    else tmem_alloc(&bars.tmem_slot, kCols);
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR == 2) cluster_sync();  // both CTAs' barriers exist before any remote arrival
  tc_fence_after();
  const uint32_t tmem = bars.tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int t = cta; t < total && ok; t += G) {
        const int b = t / per_u, rem = t % per_u;
        const int mt = PAIR * (rem / n_tiles) + rank, nt = rem % n_tiles;
        const long long a0 = p.a + b * p.a_batch + (long long)mt * p.kt;
        const long long b0 = p.b + b * p.b_batch + (long long)nt * C::kBTiles * p.kt;
        for (int h = 0; h < 2 * p.kt; ++h, ++it) {  // half tiles: kt = h / 2, core columns 4 (h % 2) .. +3
          const int s = it % C::kStages;
          const uint32_t ph = (it / C::kStages) & 1;
          if (!mbar_wait(&empty[s], ph ^ 1, abort_flag)) { ok = false; break; }
          unsigned char* st = smem + s * kStageBytes;
          const int kt = h >> 1, kc = 4 * (h & 1);
          if constexpr (PAIR == 2) {
            // both CTAs' copies complete on the even CTA's barrier, which
            // expects the bytes of both
            const uint32_t fb = cluster_addr(&full[s], 0);
            if (rank == 0) mbar_arrive_expect_tx(&full[s], 2 * kStageBytes);
            for (int sa = 0; sa < C::kSa; ++sa)
              tma_load_4d_pair(&p.map, st + sa * C::kHalfBytes, 0, kc, 0, (int)(a0 + sa * p.a_slice + kt), fb);
            for (int sb = 0; sb < C::kSb; ++sb)
              tma_load_4d_pair(&p.map, st + (C::kSa + sb) * C::kHalfBytes, 0, kc, 0,
                               (int)(b0 + sb * p.b_slice + (long long)rank * p.kt + kt), fb);
          } else {
            mbar_arrive_expect_tx(&full[s], kStageBytes);
            for (int sa = 0; sa < C::kSa; ++sa)
              tma_load_4d(&p.map, st + sa * C::kHalfBytes, 0, kc, 0, (int)(a0 + sa * p.a_slice + kt), &full[s]);
            for (int sb = 0; sb < C::kSb; ++sb)
              for (int u = 0; u < C::kBTiles; ++u)
                tma_load_4d(&p.map, st + (C::kSa + sb * C::kBTiles + u) * C::kHalfBytes, 0, kc, 0,
                            (int)(b0 + sb * p.b_slice + (long long)u * p.kt + kt), &full[s]);
          }
        }
      }
      // no copy may be left in flight at exit: the even CTA (or a single one)
      // waits for its stages to fill, the odd CTA of a pair, whose copies
      // complete on the even CTA's barrier, for its stages to be released by
      // the products (one bounded budget in all)
      const uint64_t t0 = global_ns();
      for (int k = it - C::kStages < 0 ? 0 : it - C::kStages; k < it; ++k) {
        uint64_t* bar = (PAIR == 2 && rank == 1) ? &empty[k % C::kStages] : &full[k % C::kStages];
        while (!mbar_test(bar, (k / C::kStages) & 1) && global_ns() - t0 < kDrainNs) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      constexpr uint32_t idesc = idesc_bf16(128 * PAIR, C::kBn);
      int it = 0, lt = 0;
      bool ok = true;
      for (int t = cta; t < total && ok; t += G, ++lt) {
        const int buf = lt & 1;
        if (lt >= 2) {
          if (!mbar_wait(&acc_empty[buf], ((lt >> 1) - 1) & 1, abort_flag)) { ok = false; break; }
          tc_fence_after();
        }
        const uint32_t d = tmem + buf * kAccCols;
        for (int h = 0; h < 2 * p.kt; ++h, ++it) {
          const int s = it % C::kStages;
          if (!mbar_wait(&full[s], (it / C::kStages) & 1, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + s * kStageBytes);
          // half tile: 4 core columns (LBO 128 B), 8-row groups 512 B apart
#pragma unroll
          for (int kk = 0; kk < kTileK / 32; ++kk) {
#pragma unroll
            for (int q = 0; q < Pairs::kPairs; ++q) {
              const uint32_t a_addr = st + Pairs::a(q) * C::kHalfBytes + kk * 256;
              const uint32_t b_addr = st + (C::kSa + Pairs::b(q) * kBPer) * C::kHalfBytes + kk * 256;
              const uint32_t acc = (h > 0 || kk > 0 || !Pairs::first(q)) ? 1u : 0u;
              const uint32_t dq = d + Pairs::acc(q) * C::kBn;
              if constexpr (PAIR == 2)
                mma_bf16_pair(dq, smem_desc(a_addr, 128, 512), smem_desc(b_addr, 128, 512), idesc, acc);
              else
                mma_bf16(dq, smem_desc(a_addr, 128, 512), smem_desc(b_addr, 128, 512), idesc, acc);
            }
          }
          if constexpr (PAIR == 2) {
            mma_commit_pair(cluster_addr(&empty[s], 0));
            mma_commit_pair(cluster_addr(&empty[s], 1));
          } else {
            mma_commit(&empty[s]);
          }
        }
        if (ok) {
          if constexpr (PAIR == 2) {
            mma_commit_pair(cluster_addr(&acc_full[buf], 0));
            mma_commit_pair(cluster_addr(&acc_full[buf], 1));
          } else {
            mma_commit(&acc_full[buf]);
          }
        }
      }
      // completes when every product issued above has (also after an abort)
      if constexpr (PAIR == 2) {
        mma_commit_pair(cluster_addr(&bars.drain, 0));
        mma_commit_pair(cluster_addr(&bars.drain, 1));
      } else {
        mma_commit(&bars.drain);
      }
    }
  } else {
    // EPIW epilogue warps: warp w owns TMEM lanes 32 (w % 4) .. +31 and one of
    // EPIW / 4 column ranges of the tile
    const int q = warp & 3;
    const int part = (warp - 2) >> 2;
    constexpr int kParts = EPIW / 4;
    constexpr int kSpan = C::kBn / kParts;
    // staging boxes start 1 KB after the barrier block (1024-byte aligned for
    // the swizzle); box k of this warp has the load barrier box_bar[k]
    unsigned char* red_stage = smem + C::kStages * kStageBytes + 1024 + (warp - 2) * kRedBuf * kRedBox;
    uint64_t* box_bar = bars.box + (warp - 2) * kRedBuf;
    uint32_t box_phase = 0;    // bit k: parity of box_bar[k]'s next completion
    uint32_t box_loading = 0;  // bit k: a load into box k is in flight
    int nred = 0;
    int lt = 0;
    bool ok = true;
    for (int t = cta; t < total && ok; t += G, ++lt) {
      const int b = t / per_u, rem = t % per_u;
      const int mt = PAIR * (rem / n_tiles) + rank, nt = rem % n_tiles;
      const int buf = lt & 1;
      const int md = epi.mode(mt, nt);
      const int row = q * 32 + lane;
      const int c_begin = part * kSpan, c_end = (part + 1) * kSpan;
      // mode 2 tiles need the old values on the SM: chunk i's 32 x 32 box is
      // loaded into box i % kRedBuf, kRedBuf chunks ahead, the first kRedBuf
      // before the accumulator wait (so their latency hides behind the products)
      auto load_box = [&](int k, int c0) {
        if constexpr (Epi::kStage) {
          if (lane == 0) {
            bulk_wait_read();  // no bulk operation still reads a box of this warp
            mbar_arrive_expect_tx(&box_bar[k], kRedBox);
            tma_load_2d(&epi.red_map, red_stage + k * kRedBox, epi.red_x(nt, c0), epi.red_y(b, mt, q * 32),
                        &box_bar[k]);
          }
          box_loading |= 1u << k;
        }
      };
      if constexpr (Epi::kStage) {
        if (md == 2)
          for (int i = 0; i < kRedBuf && c_begin + 32 * i < c_end; ++i) load_box(i, c_begin + 32 * i);
      }
      // waits are made warp-uniform: the loop below issues .sync.aligned loads
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (lt >> 1) & 1, abort_flag))) break;
      tc_fence_after();
#pragma unroll 1
      for (int c0 = c_begin; c0 < c_end; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + buf * kAccCols + c0, v);
        if constexpr (Pairs::kAccs == 2) {
          float v2[32];  // the same columns of the second accumulator
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + buf * kAccCols + C::kBn + c0, v2);
          epi(b, mt, nt, row, c0, v, v2);
        } else if constexpr (Epi::kStage) {
          const int ci = (c0 - c_begin) >> 5;  // chunk index within this warp's columns
          const int k = md == 2 ? ci % kRedBuf : nred % kRedBuf;
          const bool keep = md == 2 && epi.keeps(mt, nt);
          unsigned char* box = red_stage + k * kRedBox;
          if (md == 2) {
            if (!__all_sync(0xffffffffu, mbar_wait(&box_bar[k], (box_phase >> k) & 1, abort_flag))) {
              ok = false;
              break;
            }
            box_phase ^= 1u << k;
            box_loading &= ~(1u << k);
            float4 o[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) o[u] = *reinterpret_cast<const float4*>(box + lane * 128 + ((u ^ (lane & 7)) << 4));
            epi.finish(b, mt, nt, row, c0, o, v);  // o: old -> new values; panels written
            __syncwarp();
            if (keep)
#pragma unroll
              for (int u = 0; u < 8; ++u)
                *reinterpret_cast<float4*>(box + lane * 128 + ((u ^ (lane & 7)) << 4)) = o[u];
            nred = k + 1;  // the next plain box follows in the ring
          } else {
            // -acc of the warp's 32 rows x 32 columns as one swizzled box
            // (row r, 16-byte chunk u at chunk u ^ (r & 7))
            if (lane == 0) bulk_wait_read_n<kRedBuf - 1>();  // the box's previous operation has read it
            __syncwarp();
#pragma unroll
            for (int u = 0; u < 8; ++u)
              *reinterpret_cast<float4*>(box + lane * 128 + ((u ^ (lane & 7)) << 4)) =
                  make_float4(-v[4 * u], -v[4 * u + 1], -v[4 * u + 2], -v[4 * u + 3]);
            ++nred;
          }
          // the box goes to the output by one tensor bulk operation: added at
          // L2 (mode 0, no load on the SM) or stored (modes 1 and 2: the old
          // values are dropped or already applied)
          fence_proxy_async();
          __syncwarp();
          if (lane == 0 && (md != 2 || keep)) {
            if (md == 0)
              tma_reduce_add_2d(&epi.red_map, box, epi.red_x(nt, c0), epi.red_y(b, mt, q * 32));
            else
              tma_store_2d(&epi.red_map, box, epi.red_x(nt, c0), epi.red_y(b, mt, q * 32));
            bulk_commit();
          }
          // the box is free again (load_box first waits for the store to read it)
          if (md == 2 && c0 + 32 * kRedBuf < c_end) load_box(k, c0 + 32 * kRedBuf);
        } else {
          epi(b, mt, nt, row, c0, v);
        }
      }
      tc_fence_before();
      if constexpr (PAIR == 2) mbar_arrive_cluster(cluster_addr(&acc_empty[buf], 0));
      else mbar_arrive(&acc_empty[buf]);
    }
    // no box load may be left in flight at exit (only after an abort)
    for (int k = 0; k < kRedBuf; ++k) {
      if (!(box_loading >> k & 1)) continue;
      const uint64_t t0 = global_ns();
      while (!mbar_test(&box_bar[k], (box_phase >> k) & 1) && global_ns() - t0 < kDrainNs) {
      }
    }
    if (Epi::kStage) bulk_wait_all();
  }
  __syncthreads();
  if (warp == 1) {
    // the tensor core must be idle before the columns are released
    const uint64_t t0 = global_ns();
    while (!mbar_test(&bars.drain, 0) && global_ns() - t0 < kDrainNs) {
    }
  }
  if constexpr (PAIR == 2) cluster_sync();  // no remote arrival into, or product reading, a CTA that has left
  if (warp == 1) {
    tc_fence_after();
    if constexpr (PAIR == 2) tmem_dealloc_pair(tmem, kCols);
    else tmem_dealloc(tmem, kCols);
  }
  if (threadIdx.x == 0 && *abort_flag && p.status) atomicCAS(p.status, 0, DS_TIMEOUT);
}

template <class C, class Pairs, int EPIW, class Epi>
int launch_gemm_persistent(const TileMapParams& p, int n_tiles, int m_tiles, int batch, const Epi& epi,
                           cudaStream_t st) {
  const dim3 block(64 + 32 * EPIW);
  const int stage_extra_single = Epi::kStage ? red_stage_bytes<C, EPIW>() : 0;
  if constexpr (C::kBTiles == 2) {
   if (m_tiles % 2 == 0) {
    // CTA pairs: clusters of two, as many as fit at once
    using CP = PairCfg<C, 6, 2>;
    constexpr int kStagePair = (CP::kSa + CP::kSb) * CP::kHalfBytes;
    const int smem_bytes = CP::kStages * kStagePair + 1024 + CP::kBarBytes + (Epi::kStage ? red_stage_bytes<CP, EPIW>() : 0);
    auto kern = umma_gemm_persistent_kernel<CP, Pairs, Epi, EPIW, 2>;
    int rc = ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem_bytes);
    int clusters = 0;
    if (!rc) rc = max_active_clusters(reinterpret_cast<const void*>(kern), block.x, smem_bytes, &clusters);
    if (rc) return rc;
    const int units = n_tiles * (m_tiles / 2) * batch;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * (units < clusters ? units : clusters));
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem_bytes;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    NED_CUDA(cudaLaunchKernelEx(&cfg, kern, p, epi, n_tiles, m_tiles, batch));
    NED_LAUNCH_CHECK("umma_gemm_persistent_kernel");
    return NEDMFT_OK;
   }
  }
  const int smem_bytes = C::kSmem + stage_extra_single;
  auto kern = umma_gemm_persistent_kernel<C, Pairs, Epi, EPIW, 1>;
  int rc = ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem_bytes);
  int sms = 0;
  if (!rc) rc = device_sm_count(&sms);
  if (rc) return rc;
  const int total = n_tiles * m_tiles * batch;
  const int grid = total < sms ? total : sms;
  kern<<<grid, block, smem_bytes, st>>>(p, epi, n_tiles, m_tiles, batch);
  NED_LAUNCH_CHECK("umma_gemm_persistent_kernel");
  return NEDMFT_OK;
}


// ------------------------------------------------------------------ epilogues

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat16 a, __nv_bfloat16 b) {
  const __nv_bfloat162 v = __halves2bfloat162(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ uint4 shfl_xor_u4(uint4 v, int m) {
  return make_uint4(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m),
                    __shfl_xor_sync(0xffffffffu, v.z, m), __shfl_xor_sync(0xffffffffu, v.w, m));
}
// Within each quad of lanes (l = lane & 3): e[p] of lane l becomes lane p's
// original e[l].  Step 1 transposes the 2 x 2 blocks of lane pairs, step 2
// swaps the off-diagonal blocks.  Every lane of the warp must take part.
__device__ __forceinline__ void quad_transpose4(uint4* e, int l) {
  const bool b1 = l & 1, b2 = (l >> 1) & 1;
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const uint4 r = shfl_xor_u4(b1 ? e[2 * g] : e[2 * g + 1], 1);
    if (b1) e[2 * g] = r; else e[2 * g + 1] = r;
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint4 r = shfl_xor_u4(b2 ? e[h] : e[2 + h], 2);
    if (b2) e[h] = r; else e[2 + h] = r;
  }
}

// A <- A(rows K and columns K zeroed) - acc, A interleaved FP32 (row stride 2
// np floats), for a Gauss-Jordan block of W complex columns (W = 128, 256).
template <int W>
struct EpiUpdate {
  static constexpr int kKtW = 2 * W / kTileK;  // K tiles of the rank-W products
  static constexpr bool kStage = true;
  float* A;
  size_t bstride;  // floats between matrices
  int np, k0;
  // the next step's panels, written from the new values (kn < 0: last step)
  int kn;
  __nv_bfloat16* cimg;  // C' of step kn (the update's A operand)
  __nv_bfloat16* timg;  // embedded A_{Kn,:}^T (the R product's B operand)
  size_t pstride, cslice, tslice;
  // 0: plain tile, A += -acc by bulk reduction at L2; 1: rows or columns of
  // block K (new value = -acc); 2: the next step's panel blocks (new values
  // needed in registers)
  // (a tile, 128 rows by 128 complex columns, lies wholly inside or outside a block)
  __device__ static bool in_block(int x, int k) { return x >= k && x < k + W; }
  __device__ int mode(int mt, int nt) const {
    if (kn >= 0 && (in_block(nt * (CfgGJ::kBn / 2), kn) || in_block(mt * kTileRows, kn))) return 2;
    if (in_block(nt * (CfgGJ::kBn / 2), k0) || in_block(mt * kTileRows, k0)) return 1;
    return 0;
  }
  // Mode 2 tiles are stored back only in the diagonal block (Kn, Kn), which
  // the next pivot reads; the rest of block row and column Kn is read only
  // through the panels written here (the next update replaces it).
  __device__ bool keeps(int mt, int nt) const {
    return in_block(nt * (CfgGJ::kBn / 2), kn) && in_block(mt * kTileRows, kn);
  }
  // A of the whole batch as one FP32 tensor of 2 np columns and batch * np
  // rows, moved in boxes of 32 x 32 with 128-byte swizzle (the staged -acc)
  CUtensorMap red_map;
  __device__ int red_x(int nt, int c0) const { return nt * CfgGJ::kBn + c0; }
  __device__ int red_y(int b, int mt, int r0) const { return b * np + mt * kTileRows + r0; }
  // mode 2 chunk of row r, real columns c0 .. c0+31 of the tile: o holds the
  // old values and gets the new ones, old - acc (old values in block K
  // dropped); the next step's panels are written from them
  __device__ void finish(int b, int mt, int nt, int r, int c0, float4* o, const float* v) const {
    const int i = mt * kTileRows + r;
    const int n0 = nt * CfgGJ::kBn + c0;  // real column
    const int j0 = n0 >> 1;               // first complex column of the chunk
    const bool skip = in_block(i, k0) || in_block(nt * (CfgGJ::kBn / 2), k0);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int ja = j0 + 2 * u;
      if (skip || in_block(ja, k0)) { o[u].x = 0.f; o[u].y = 0.f; }
      if (skip || in_block(ja + 1, k0)) { o[u].z = 0.f; o[u].w = 0.f; }
      o[u].x -= v[4 * u]; o[u].y -= v[4 * u + 1]; o[u].z -= v[4 * u + 2]; o[u].w -= v[4 * u + 3];
    }
    if (kn < 0) return;
    if (in_block(nt * (CfgGJ::kBn / 2), kn)) {
      // column block Kn: row i of C'_next (C'_Kn = -I)
      // 4 complex values = one 16-byte core-matrix row per slice
      __nv_bfloat16* cd = cimg + b * pstride;
      const bool in = in_block(i, kn);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int u = 4 * g + e;
          const int c = j0 + u - kn;
          float re = (u & 1) ? o[u >> 1].z : o[u >> 1].x;
          float im = (u & 1) ? o[u >> 1].w : o[u >> 1].y;
          if (in) { re = (i - kn == c) ? -1.f : 0.f; im = 0.f; }
          __nv_bfloat16 rh, rl, ih, il;
          split2(re, rh, rl);
          split2(im, ih, il);
          const __nv_bfloat162 h2 = __halves2bfloat162(rh, ih), l2 = __halves2bfloat162(rl, il);
          hi[e] = *reinterpret_cast<const uint32_t*>(&h2);
          lo[e] = *reinterpret_cast<const uint32_t*>(&l2);
        }
        const size_t off = img_offset(i, 2 * (j0 + 4 * g - kn), kKtW);  // 8-element aligned
        *reinterpret_cast<uint4*>(cd + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(cd + cslice + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
    if (in_block(mt * kTileRows, kn)) {
      // row block Kn: row c = i - kn of A_{Kn,:} (A_{Kn,Kn} -> I) as (Re, Im)
      // pairs over k: column j gives row j of the image at k = 2c, 2c+1.  A
      // 16-byte core-matrix row holds k = 2c .. 2c+7 of one row, i.e. 4
      // consecutive c: each quad of lanes transposes its values (a 4 x 4
      // transpose of 16-byte elements in two xor exchanges) so that lane l of
      // the quad writes whole rows of column j0 + 4 jq + l.
      __nv_bfloat16* td = timg + b * pstride;
      const int c = i - kn;
      const int l = r & 3;
      const int cq = c - l;
#pragma unroll
      for (int jq = 0; jq < 4; ++jq) {
        uint4 e[4];  // e[p]: (hi, lo) at k = 2c of column j = j0 + 4 jq + p
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const int u = 4 * jq + p;
          const int j = j0 + u;
          float re = (u & 1) ? o[u >> 1].z : o[u >> 1].x;
          float im = (u & 1) ? o[u >> 1].w : o[u >> 1].y;
          if (in_block(j, kn)) { re = (j - kn == c) ? 1.f : 0.f; im = 0.f; }
          __nv_bfloat16 rh, rl, ih, il;
          split2(re, rh, rl);
          split2(im, ih, il);
          e[p] = make_uint4(bf2_bits(rh, ih), bf2_bits(rl, il), 0u, 0u);
        }
        quad_transpose4(e, l);  // e[m]: lane m's element for p = l
        const int j = j0 + 4 * jq + l;
        const size_t o0 = img_offset(j, 2 * cq, kKtW);
        *reinterpret_cast<uint4*>(td + o0) = make_uint4(e[0].x, e[1].x, e[2].x, e[3].x);
        *reinterpret_cast<uint4*>(td + tslice + o0) = make_uint4(e[0].y, e[1].y, e[2].y, e[3].y);
      }
    }
  }
};

// R (W x np complex; accumulator 0 = Re R, 1 = Im R, rows = R rows, columns
// = complex columns j) -> the update's B operand image: rows n = 2j, 2j+1;
// k = 2r, 2r+1 with [[re, -im], [im, re]].
template <int W>
struct EpiRPack {
  static constexpr bool kStage = false;
  static constexpr int kKtW = 2 * W / kTileK;
  static constexpr int kBn = 128;  // complex columns per tile
  __device__ int mode(int, int) const { return 1; }
  __nv_bfloat16* img;   // per matrix: 2 slices x (2 np x 2 W)
  size_t bstride;       // elements between matrices
  size_t slice;         // elements between slices
  // row r of R, complex columns j0 .. j0+31: rows 2j, 2j+1 of the image at
  // k = 2r, 2r+1; a quad of lanes (4 consecutive r) exchanges its values so
  // that each lane writes whole 16-byte core-matrix rows (see EpiUpdate's
  // A_K panel)
  __device__ void operator()(int b, int mt, int nt, int r_tile, int c0, const float* re_v,
                             const float* im_v) const {
    __nv_bfloat16* base = img + b * bstride;
    const int r = mt * kTileRows + r_tile;  // row of R
    const int l = r_tile & 3, rq = r - l;
    const int j0 = nt * kBn + c0;
#pragma unroll
    for (int jq = 0; jq < 8; ++jq) {
      uint4 e[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int u = 4 * jq + p;
        const float re = re_v[u], im = im_v[u];
        __nv_bfloat16 rh, rl, ih, il, nh, nl;
        split2(re, rh, rl);
        split2(im, ih, il);
        split2(-im, nh, nl);
        e[p] = make_uint4(bf2_bits(rh, nh), bf2_bits(ih, rh), bf2_bits(rl, nl), bf2_bits(il, rl));
      }
      quad_transpose4(e, l);
      const int j = j0 + 4 * jq + l;
      const size_t o0 = img_offset(2 * j, 2 * rq, kKtW), o1 = img_offset(2 * j + 1, 2 * rq, kKtW);
      *reinterpret_cast<uint4*>(base + o0) = make_uint4(e[0].x, e[1].x, e[2].x, e[3].x);
      *reinterpret_cast<uint4*>(base + o1) = make_uint4(e[0].y, e[1].y, e[2].y, e[3].y);
      *reinterpret_cast<uint4*>(base + slice + o0) = make_uint4(e[0].z, e[1].z, e[2].z, e[3].z);
      *reinterpret_cast<uint4*>(base + slice + o1) = make_uint4(e[0].w, e[1].w, e[2].w, e[3].w);
    }
  }
};

// ------------------------------------------------------------------ panel kernels (CUDA cores)


// P = inv(A_KK) (kNb x kNb, FP32, no pivoting -- the static row order makes
// the pivots safe) written as the R-product's A operand (P' and P'', row r,
// k = 2c / 2c+1).
// A_KK sits in shared memory and is inverted in two 64-column halves (block
// Gauss-Jordan):
//   B11 <- P1 = inv(A11);  B12 <- P1 A12;  B22 <- A22 - A21 B12;  B21 <- -A21 P1;
//   B22 <- X22 = inv(B22); V = -B12 X22;  B21 <- X22 B21;  B11 <- P1 + V B21(old);  B12 <- V,
// the two 64 x 64 inversions unblocked (one barrier per pivot, 2 x 2 complex
// entries per thread), the products by two halves of 512 threads (4 x 2
// outputs each).
constexpr int kPivH = kNb / 2;
constexpr size_t kPivSmem = (size_t)(kNb * kNb + kPivH * kPivH) * sizeof(float2);  // 160 KB

struct alignas(16) PivShared {
  float4 rowb[2][2][kPivH / 2];  // [buffer][pivot row][column pair]
  float4 colb[2][kPivH];         // [buffer][row]: the row's two entries in the pivot columns
  float4 pivb[2][2];             // [buffer][row of P^-1]
  int bad;
};

__device__ __forceinline__ float2 shfl_c(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// unblocked in-place Gauss-Jordan of the 64 x 64 block of M (row stride kNb) at (o, o),
// two pivots per barrier: thread (warp w, lane l) holds rows 2w, 2w+1 x columns 2l, 2l+1,
// so step s eliminates with the 2 x 2 pivot block P held by thread (s, s) (P^-1 by
// two scalar pivots: p11 and the Schur complement p22 - p21 p11^-1 p12).  Warp s
// broadcasts its rows A_K with the pivot columns replaced by the identity and turns
// them into P^-1 A_K (P^-1 in the pivot columns); every other row r takes
// a[r][c] <- [c not a pivot column] a[r][c] - g_r rowb[:, c] with g_r = a[r][K] P^-1
// (so its pivot columns become -g_r).
__device__ __forceinline__ void piv_gj64(float2* M, int o, PivShared& sh) {
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int rr = 2 * w, cc = 2 * lane;
  float2 a[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) a[i][j] = M[(o + rr + i) * kNb + o + cc + j];
  for (int s = 0; s < kPivH / 2; ++s) {
    const int buf = s & 1;
    if (lane == s)  // the rows' entries in the pivot columns, before the step
#pragma unroll
      for (int i = 0; i < 2; ++i)
        sh.colb[buf][rr + i] = make_float4(a[i][0].x, a[i][0].y, a[i][1].x, a[i][1].y);
    if (w == s) {  // warp-uniform: the pivot rows
      float2 q00 = make_float2(0.f, 0.f), q01 = q00, q10 = q00, q11 = q00;
      if (lane == s) {
        float2 i1, is;
        const bool ok1 = cinv_guard<float>(a[0][0], i1, 1e-6f);
        const float2 t12 = cmul(i1, a[0][1]);  // p11^-1 p12
        const float2 t21 = cmul(a[1][0], i1);  // p21 p11^-1
        const bool ok2 = cinv_guard<float>(csub(a[1][1], cmul(a[1][0], t12)), is, 1e-6f);
        if (!ok1 || !ok2) sh.bad = 1;
        const float2 u = cmul(t12, is);
        q00 = cadd(i1, cmul(u, t21));
        q01 = make_float2(-u.x, -u.y);
        const float2 v = cmul(is, t21);
        q10 = make_float2(-v.x, -v.y);
        q11 = is;
        sh.pivb[buf][0] = make_float4(q00.x, q00.y, q01.x, q01.y);
        sh.pivb[buf][1] = make_float4(q10.x, q10.y, q11.x, q11.y);
      }
      q00 = shfl_c(q00, s);
      q01 = shfl_c(q01, s);
      q10 = shfl_c(q10, s);
      q11 = shfl_c(q11, s);
      float2 r0[2], r1[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        r0[j] = cadd(cmul(q00, a[0][j]), cmul(q01, a[1][j]));
        r1[j] = cadd(cmul(q10, a[0][j]), cmul(q11, a[1][j]));
      }
      if (lane == s) {
        sh.rowb[buf][0][lane] = make_float4(1.f, 0.f, 0.f, 0.f);
        sh.rowb[buf][1][lane] = make_float4(0.f, 0.f, 1.f, 0.f);
        a[0][0] = q00; a[0][1] = q01;
        a[1][0] = q10; a[1][1] = q11;
      } else {
        sh.rowb[buf][0][lane] = make_float4(a[0][0].x, a[0][0].y, a[0][1].x, a[0][1].y);
        sh.rowb[buf][1][lane] = make_float4(a[1][0].x, a[1][0].y, a[1][1].x, a[1][1].y);
        a[0][0] = r0[0]; a[0][1] = r0[1];
        a[1][0] = r1[0]; a[1][1] = r1[1];
      }
    }
    __syncthreads();
    if (w != s) {
      const float4 p0 = sh.pivb[buf][0], p1 = sh.pivb[buf][1];
      const float4 b0 = sh.rowb[buf][0][lane], b1 = sh.rowb[buf][1][lane];
      const float2 rk0[2] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w)};
      const float2 rk1[2] = {make_float2(b1.x, b1.y), make_float2(b1.z, b1.w)};
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const float4 c4 = sh.colb[buf][rr + i];
        const float2 x0 = make_float2(c4.x, c4.y), x1 = make_float2(c4.z, c4.w);
        // g = (x0, x1) P^-1
        const float2 g0 = cadd(cmul(x0, make_float2(p0.x, p0.y)), cmul(x1, make_float2(p1.x, p1.y)));
        const float2 g1 = cadd(cmul(x0, make_float2(p0.z, p0.w)), cmul(x1, make_float2(p1.z, p1.w)));
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          float2 v = lane == s ? make_float2(0.f, 0.f) : a[i][j];
          v.x -= g0.x * rk0[j].x - g0.y * rk0[j].y + g1.x * rk1[j].x - g1.y * rk1[j].y;
          v.y -= g0.x * rk0[j].y + g0.y * rk0[j].x + g1.x * rk1[j].y + g1.y * rk1[j].x;
          a[i][j] = v;
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) M[(o + rr + i) * kNb + o + cc + j] = a[i][j];
}

// acc[a][c] = sum_{k0 <= k < k0 + kn} X[i0 + a][k] Y[k][j0 + c] (a < 4, c < 2)
// for the 4 x 2 block of thread s (0 .. 511) of a 64 x 64 product (row
// strides ldx, ldy): i0 = 4 (s / 32), j0 = 2 (s % 32), so a warp reads one X
// entry per row (a broadcast) and one 512-byte row of Y per k.
__device__ __forceinline__ void piv_mm(const float2* X, int ldx, const float2* Y, int ldy, int s, int k0, int kn,
                                       float2 (&acc)[4][2]) {
  const int i0 = 4 * (s >> 5), j0 = 2 * (s & 31);
#pragma unroll
  for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = make_float2(0.f, 0.f);
#pragma unroll 4
  for (int k = k0; k < k0 + kn; ++k) {
    const float4 y = *reinterpret_cast<const float4*>(Y + k * ldy + j0);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float2 x = X[(i0 + a) * ldx + k];
      acc[a][0].x += x.x * y.x - x.y * y.y;
      acc[a][0].y += x.x * y.y + x.y * y.x;
      acc[a][1].x += x.x * y.z - x.y * y.w;
      acc[a][1].y += x.x * y.w + x.y * y.z;
    }
  }
}
__device__ __forceinline__ void piv_put(float2* Z, int ldz, int s, const float2 (&v)[4][2]) {
  const int i0 = 4 * (s >> 5), j0 = 2 * (s & 31);
#pragma unroll
  for (int a = 0; a < 4; ++a)
    *reinterpret_cast<float4*>(Z + (i0 + a) * ldz + j0) = make_float4(v[a][0].x, v[a][0].y, v[a][1].x, v[a][1].y);
}
// v += sign * Z (the thread's 4 x 2 block)
__device__ __forceinline__ void piv_acc(const float2* Z, int ldz, int s, float sign, float2 (&v)[4][2]) {
  const int i0 = 4 * (s >> 5), j0 = 2 * (s & 31);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float4 z = *reinterpret_cast<const float4*>(Z + (i0 + a) * ldz + j0);
    v[a][0].x += sign * z.x; v[a][0].y += sign * z.y;
    v[a][1].x += sign * z.z; v[a][1].y += sign * z.w;
  }
}
__device__ __forceinline__ void piv_neg(float2 (&v)[4][2]) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) v[a][c] = make_float2(-v[a][c].x, -v[a][c].y);
}

// Four entries z[0..3] of a row of P (consecutive columns) as the R
// product's A operand: a 16-byte core-matrix row of each of the four slices,
// P' = (Re P, -Im P) hi, lo and P'' = (Im P, Re P) hi, lo, `slice` apart.
__device__ __forceinline__ void piv_store4(__nv_bfloat16* dst, size_t slice, size_t o, const float2 (&z)[4]) {
  uint32_t h1[4], l1[4], h2[4], l2[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __nv_bfloat16 rh, rl, ih, il, nh, nl;
    split2(z[q].x, rh, rl);
    split2(z[q].y, ih, il);
    split2(-z[q].y, nh, nl);
    h1[q] = bf2_bits(rh, nh);
    l1[q] = bf2_bits(rl, nl);
    h2[q] = bf2_bits(ih, rh);
    l2[q] = bf2_bits(il, rl);
  }
  *reinterpret_cast<uint4*>(dst + o) = make_uint4(h1[0], h1[1], h1[2], h1[3]);
  *reinterpret_cast<uint4*>(dst + slice + o) = make_uint4(l1[0], l1[1], l1[2], l1[3]);
  *reinterpret_cast<uint4*>(dst + 2 * slice + o) = make_uint4(h2[0], h2[1], h2[2], h2[3]);
  *reinterpret_cast<uint4*>(dst + 3 * slice + o) = make_uint4(l2[0], l2[1], l2[2], l2[3]);
}

__global__ void __launch_bounds__(1024) gj_pivot_pack_kernel(const float2* __restrict__ A, int np, int k0,
                                                             __nv_bfloat16* __restrict__ pimg, size_t pstride,
                                                             size_t pslice, int* status) {
  extern __shared__ __align__(16) float2 piv_smem[];
  __shared__ PivShared sh;
  float2* M = piv_smem;               // A_KK, row stride kNb
  float2* T = piv_smem + kNb * kNb;   // 64 x 64 temporary
  float2* B11 = M;
  float2* B12 = M + kPivH;
  float2* B21 = M + kPivH * kNb;
  float2* B22 = M + kPivH * kNb + kPivH;
  const int b = blockIdx.x;
  const int t = threadIdx.x;
  const float2* src = A + (size_t)b * np * np;
  for (int e = t; e < kNb * kNb / 2; e += blockDim.x) {
    const int r = e / (kNb / 2), v = e % (kNb / 2);
    *reinterpret_cast<float4*>(M + r * kNb + 2 * v) =
        *reinterpret_cast<const float4*>(src + (size_t)(k0 + r) * np + k0 + 2 * v);
  }
  if (t == 0) sh.bad = 0;
  __syncthreads();
  // two halves of 512 threads: a product alone is split along K (the upper
  // half's partial sums pass through T), two independent products run side by side
  const int half = t >> 9, s = t & 511;
  float2 u[4][2];
  piv_gj64(M, 0, sh);  // B11 <- P1
  __syncthreads();
  piv_mm(B11, kNb, B12, kNb, s, 32 * half, 32, u);  // P1 A12
  if (half) piv_put(T, kPivH, s, u);
  __syncthreads();
  if (!half) {
    piv_acc(T, kPivH, s, 1.f, u);
    piv_put(B12, kNb, s, u);  // B12 <- P1 A12
  }
  __syncthreads();
  piv_mm(B21, kNb, half ? B11 : B12, kNb, s, 0, kPivH, u);  // A21 B12 | A21 P1
  __syncthreads();
  if (!half) {
    piv_neg(u);
    piv_acc(B22, kNb, s, 1.f, u);
    piv_put(B22, kNb, s, u);  // B22 <- A22 - A21 B12
  } else {
    piv_neg(u);
    piv_put(B21, kNb, s, u);  // B21 <- -A21 P1
  }
  __syncthreads();
  piv_gj64(M, kPivH, sh);  // B22 <- X22
  __syncthreads();
  piv_mm(B12, kNb, B22, kNb, s, 32 * half, 32, u);  // B12 X22
  if (half) piv_put(T, kPivH, s, u);
  __syncthreads();
  if (!half) {
    piv_acc(T, kPivH, s, 1.f, u);
    piv_neg(u);
    piv_put(T, kPivH, s, u);  // V = -B12 X22
  }
  __syncthreads();
  piv_mm(half ? T : B22, half ? kPivH : kNb, B21, kNb, s, 0, kPivH, u);  // X22 B21 | V B21
  __syncthreads();
  if (!half) {
    piv_put(B21, kNb, s, u);  // B21 <- X22 B21
    float2 v[4][2] = {};
    piv_acc(T, kPivH, s, 1.f, v);
    piv_put(B12, kNb, s, v);  // B12 <- V
  } else {
    piv_acc(B11, kNb, s, 1.f, u);
    piv_put(B11, kNb, s, u);  // B11 <- P1 + V B21
  }
  __syncthreads();
  if (sh.bad && t == 0 && status) atomicCAS(status, 0, DS_SINGULAR);
  // row r, k = 2c .. 2c + 31 for c = 16 g .. 16 g + 15: four 16-byte core-matrix rows per slice
  __nv_bfloat16* dst = pimg + b * pstride;
  {
    const int r = t >> 3, cg = 16 * (t & 7);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      float2 z[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) z[q] = M[r * kNb + cg + 4 * h + q];
      piv_store4(dst, pslice, img_offset(r, 2 * (cg + 4 * h), kKt), z);
    }
  }
}

// Copy of the W x W diagonal block A_KK of every matrix (inverted in place by
// the W = 128 Gauss-Jordan when the outer block is wider).  Block (x, y): rows
// 8x .. 8x+7 of matrix y, two entries (16 bytes) per thread and step.
constexpr int kPackRows = 8;
template <int W>
__global__ void __launch_bounds__(256) gj_extract_kernel(const float2* __restrict__ A, int np, int k0,
                                                         float2* __restrict__ out) {
  const int b = blockIdx.y, r0 = blockIdx.x * kPackRows;
  for (int e = threadIdx.x; e < kPackRows * W / 2; e += blockDim.x) {
    const int r = r0 + e / (W / 2), c = 2 * (e % (W / 2));
    const float4 v = *reinterpret_cast<const float4*>(A + (size_t)b * np * np + (size_t)(k0 + r) * np + k0 + c);
    *reinterpret_cast<float4*>(out + ((size_t)b * W + r) * W + c) = v;
  }
}

// P = inv(A_KK) (W x W, FP32) as the R-product's A operand (P' and P'' hi,
// lo: row r, k = 2c / 2c+1).  Block (x, y): rows 8x .. 8x+7 of matrix y (one 8-row group); a
// thread takes 4 consecutive entries, one 16-byte core-matrix row per slice,
// and 8 consecutive threads the 8 rows of one 128-byte core matrix.
template <int W>
__global__ void __launch_bounds__(256) gj_ppack_kernel(const float2* __restrict__ Pinv, __nv_bfloat16* __restrict__ pimg,
                                                       size_t pstride, size_t pslice) {
  static_assert(kPackRows == 8, "one core-matrix row group per block");
  const int b = blockIdx.y, r0 = blockIdx.x * kPackRows;
  __nv_bfloat16* dst = pimg + b * pstride;
  for (int e = threadIdx.x; e < kPackRows * W / 4; e += blockDim.x) {
    const int r = r0 + (e & 7), c4 = 4 * (e >> 3);
    const float4* src = reinterpret_cast<const float4*>(Pinv + ((size_t)b * W + r) * W + c4);
    const float4 z01 = src[0], z23 = src[1];
    const float2 z[4] = {make_float2(z01.x, z01.y), make_float2(z01.z, z01.w), make_float2(z23.x, z23.y),
                         make_float2(z23.z, z23.w)};
    piv_store4(dst, pslice, img_offset(r, 2 * c4, 2 * W / kTileK), z);
  }
}

// Block x of matrix y: rows x*128 .. +127 of C' (the update's A operand) and
// columns x*128 .. +127 of A_{K,:}^T as (Re, Im) pairs over k (the R-product's
// B operand),
// for a block K of W columns.  A thread takes 4 consecutive columns c of C'
// (one 16-byte core-matrix row per slice) or 4 consecutive rows c of A_{K,:}
// at one column j (consecutive threads: consecutive j, coalesced loads).
template <int W>
__global__ void __launch_bounds__(256) gj_panel_pack_kernel(const float2* __restrict__ A, int np, int k0,
                                                            __nv_bfloat16* __restrict__ cimg, size_t cstride,
                                                            size_t cslice, __nv_bfloat16* __restrict__ timg,
                                                            size_t tstride, size_t tslice) {
  constexpr int kKtW = 2 * W / kTileK;
  constexpr int G = W / 4;
  const int b = blockIdx.y;
  const int base = blockIdx.x * 128;
  const float2* src = A + (size_t)b * np * np;
  __nv_bfloat16* cd = cimg + b * cstride;
  __nv_bfloat16* td = timg + b * tstride;
  for (int e = threadIdx.x; e < 128 * G; e += blockDim.x) {
    {  // C'[i][c4 .. c4+3]; a warp covers 8 rows x 4 cores (4 contiguous 128-byte core matrices)
      const int grp = e >> 5;
      const int i = base + (grp & 15) * 8 + (e & 7);
      const int c4 = 4 * ((grp >> 4) * 4 + ((e >> 3) & 3));
      const bool in = (i >= k0 && i < k0 + W);
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 z = in ? make_float2(i - k0 == c4 + q ? -1.f : 0.f, 0.f) : src[(size_t)i * np + k0 + c4 + q];
        __nv_bfloat16 rh, rl, ih, il;
        split2(z.x, rh, rl);
        split2(z.y, ih, il);
        hi[q] = bf2_bits(rh, ih);
        lo[q] = bf2_bits(rl, il);
      }
      const size_t o = img_offset(i, 2 * c4, kKtW);
      *reinterpret_cast<uint4*>(cd + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(cd + cslice + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    {  // T row j at k = 2 c4 .. 2 c4 + 7: (Re, Im) of A_{K,:}[c4 .. c4+3][j]
      const int j = base + (e & 127), c4 = 4 * (e >> 7);
      const bool in = (j >= k0 && j < k0 + W);
      uint32_t h0[4], l0[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 z = in ? make_float2(j - k0 == c4 + q ? 1.f : 0.f, 0.f) : src[(size_t)(k0 + c4 + q) * np + j];
        __nv_bfloat16 rh, rl, ih, il;
        split2(z.x, rh, rl);
        split2(z.y, ih, il);
        h0[q] = bf2_bits(rh, ih);
        l0[q] = bf2_bits(rl, il);
      }
      const size_t o0 = img_offset(j, 2 * c4, kKtW);
      *reinterpret_cast<uint4*>(td + o0) = make_uint4(h0[0], h0[1], h0[2], h0[3]);
      *reinterpret_cast<uint4*>(td + tslice + o0) = make_uint4(l0[0], l0[1], l0[2], l0[3]);
    }
  }
}

// ------------------------------------------------------------------ buffer layout per matrix

struct GjBuffers {
  // bytes per matrix, each 1024-aligned; cimg / timg hold two panels each;
  // inner: for W = 256, the copy of A_KK and the W = 128 scratch that inverts it
  size_t mat, pimg, cimg, timg, rimg, inner, scratch, total;
};

size_t align1k(size_t x) { return (x + 1023) & ~(size_t)1023; }
// the packed panels start at 16 KB boundaries (tile units of the operand tensor map)
size_t align16k(size_t x) { return (x + 16383) & ~(size_t)16383; }

template <int W>
GjBuffers gj_buffers(int np) {
  GjBuffers g{};
  g.mat = align16k(sizeof(float2) * (size_t)np * np);
  g.pimg = align16k(4 * sizeof(__nv_bfloat16) * (size_t)W * 2 * W);           // P', P'' hi / lo
  g.cimg = 2 * align16k(2 * sizeof(__nv_bfloat16) * (size_t)np * 2 * W);      // C' hi / lo, two panels
  g.timg = 2 * align16k(2 * sizeof(__nv_bfloat16) * (size_t)np * 2 * W);      // A_K^T hi / lo, two panels
  g.rimg = align16k(2 * sizeof(__nv_bfloat16) * (size_t)2 * np * 2 * W);      // R embedded hi / lo
  if constexpr (W > 128) {
    const GjBuffers in = gj_buffers<128>(W);
    g.inner = in.mat + in.scratch;
  }
  g.scratch = g.pimg + g.cimg + g.timg + g.rimg + g.inner;
  g.total = g.mat + g.scratch;
  return g;
}

// Block width of the tensor-core Gauss-Jordan for padded size np: `width`
// 128 or 256 if the caller chose one (256 needs np a multiple of 256, from
// 512 up), else 256 where it fits and 128 below.
int gj_width(int np, int width) {
  const bool w256 = np >= 512 && np % 256 == 0;
  if (width == 128) return 128;
  return w256 ? 256 : 128;
}

GjBuffers gj_buffers_for(int np, int width) {
  return gj_width(np, width) == 256 ? gj_buffers<256>(np) : gj_buffers<128>(np);
}

}  // namespace

// Gauss-Jordan inversion of nb matrices (np x np FP32 complex, batch stride
// np*np, np a multiple of 128) on the tensor cores, in blocks of W = 128 or
// 256 columns (256 for np >= 512 and a multiple of 256).  `scratch` holds
// gj_buffers_for(np).scratch bytes per matrix.
namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the CUDA driver's tensor-map encoder, looked up once (no link against libcuda)
EncodeTiledFn encode_tiled_fn() {
  static const EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// Tensor map of an FP32 matrix of `rows` rows of `cols` contiguous elements,
// moved in boxes of box_cols x box_rows.
int encode_f32_rows(CUtensorMap* map, float* base, uint64_t cols, uint64_t rows, uint32_t box_cols, uint32_t box_rows,
                    CUtensorMapSwizzle swizzle) {
  const EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return set_error(NEDMFT_ECUDA, "cuTensorMapEncodeTiled is not available from the CUDA driver");
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * sizeof(float)};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t elem_strides[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, elem_strides,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(NEDMFT_ECUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
  return NEDMFT_OK;
}

}  // namespace

namespace {

// 4-D tensor map over `tiles` packed 128 x 64 bf16 tiles (16 KB each) at
// `base`, moved in half tiles: box (64 elements, 4 core columns, 16 row groups, 1).
int encode_tile_map(CUtensorMap* map, void* base, uint64_t tiles) {
  const EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return set_error(NEDMFT_ECUDA, "cuTensorMapEncodeTiled is not available from the CUDA driver");
  const cuuint64_t dims[4] = {64, 8, 16, tiles};
  const cuuint64_t strides[3] = {128, 1024, 16384};
  const cuuint32_t box[4] = {64, 4, 16, 1};
  const cuuint32_t elem_strides[4] = {1, 1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, elem_strides,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(NEDMFT_ECUDA, "cuTensorMapEncodeTiled (tiles) failed (CUresult %d)", (int)r);
  return NEDMFT_OK;
}

template <int W>
int gj_blocked_umma_w(float2* A, int n, int np, int nb, char* scratch, int* status, cudaStream_t st,
                      bool instrument) {
  if (np % W) return set_error(NEDMFT_EINVAL, "gj_blocked_umma: np=%d not a multiple of %d", np, W);
  constexpr int kKtW = 2 * W / kTileK;
  const GjBuffers g = gj_buffers<W>(np);
  // per matrix b: scratch + b * per holds its pimg | cimg | timg | rimg;
  // after the nb of those, the inner regions (W = 256)
  const size_t per = g.pimg + g.cimg + g.timg + g.rimg;
  __nv_bfloat16* pimg = reinterpret_cast<__nv_bfloat16*>(scratch);
  __nv_bfloat16* cimg = reinterpret_cast<__nv_bfloat16*>(scratch + g.pimg);
  __nv_bfloat16* timg = reinterpret_cast<__nv_bfloat16*>(scratch + g.pimg + g.cimg);
  __nv_bfloat16* rimg = reinterpret_cast<__nv_bfloat16*>(scratch + g.pimg + g.cimg + g.timg);
  const size_t pstride = per / 2, pslice = (size_t)W * 2 * W;
  const size_t cslice = (size_t)np * 2 * W;
  const size_t tslice = (size_t)np * 2 * W;
  const size_t rslice = (size_t)2 * np * 2 * W;
  // the C' / A_K^T panels alternate between two buffers: step k reads buffer
  // k & 1 while its update writes step k+1's panels into the other one
  const size_t chalf = g.cimg / 2 / sizeof(__nv_bfloat16), thalf = g.timg / 2 / sizeof(__nv_bfloat16);
  // A of the whole batch as one tensor of 2 np FP32 columns and nb np rows,
  // for the update's staged bulk reductions and box loads
  CUtensorMap red_map, tile_map;
  {
    float* a = reinterpret_cast<float*>(A);
    const uint64_t cols = 2 * (uint64_t)np, rows = (uint64_t)nb * np;
    int rc = encode_f32_rows(&red_map, a, cols, rows, 32, 32, CU_TENSOR_MAP_SWIZZLE_128B);
    // the panels of the batch as packed tiles, for the products' operand loads
    if (!rc) rc = encode_tile_map(&tile_map, scratch, per * nb / kTileBytes);
    if (rc) return rc;
  }
  // tile index (16 KB units from scratch) of an image pointer
  auto tile_of = [&](const __nv_bfloat16* ptr) {
    return (long long)((reinterpret_cast<const char*>(ptr) - scratch) / kTileBytes);
  };
  const long long per_t = (long long)(per / kTileBytes);
  gj_panel_pack_kernel<W>
      <<<dim3(np / 128, nb), 256, 0, st>>>(A, np, 0, cimg, pstride, cslice, timg, pstride, tslice);
  NED_LAUNCH_CHECK("gj_panel_pack_kernel");
  for (int k0 = 0, step = 0; k0 < np; k0 += W, ++step) {
    __nv_bfloat16* cur_c = cimg + (step & 1) * chalf;
    __nv_bfloat16* cur_t = timg + (step & 1) * thalf;
    __nv_bfloat16* nxt_c = cimg + ((step + 1) & 1) * chalf;
    __nv_bfloat16* nxt_t = timg + ((step + 1) & 1) * thalf;
    if constexpr (W == 128) {
      if (int rc = ensure_dyn_smem(reinterpret_cast<const void*>(gj_pivot_pack_kernel), (int)kPivSmem)) return rc;
      gj_pivot_pack_kernel<<<nb, 1024, kPivSmem, st>>>(A, np, k0, pimg, pstride, pslice, status);
      NED_LAUNCH_CHECK("gj_pivot_pack_kernel");
    } else {
      // P = inv(A_KK): the W = 128 Gauss-Jordan on copies of the diagonal blocks
      char* inner = scratch + per * nb;
      float2* Xs = reinterpret_cast<float2*>(inner);
      char* inner_scratch = inner + gj_buffers<128>(W).mat * nb;
      gj_extract_kernel<W><<<dim3(W / kPackRows, nb), 256, 0, st>>>(A, np, k0, Xs);
      NED_LAUNCH_CHECK("gj_extract_kernel");
      int rc = gj_blocked_umma_w<128>(Xs, W, W, nb, inner_scratch, status, st, false);
      if (rc) return rc;
      gj_ppack_kernel<W><<<dim3(W / kPackRows, nb), 256, 0, st>>>(Xs, pimg, pstride, pslice);
      NED_LAUNCH_CHECK("gj_ppack_kernel");
    }
    {  // Re R = P' A_K, Im R = P'' A_K: W x np each, K = 2W
      TileMapParams p{tile_map, tile_of(pimg), per_t, (long long)(pslice / kTileElems),
                      tile_of(cur_t), per_t, (long long)(tslice / kTileElems), kKtW, status};
      EpiRPack<W> epi{rimg, pstride, rslice};
      int rc = launch_gemm_persistent<CfgRP, Split3x2, 4>(p, np / EpiRPack<W>::kBn, W / kTileRows, nb, epi, st);
      if (rc) return rc;
    }
    {  // A <- A - C' R, np x 2np, K = 2W; next step's panels from the epilogue
      TileMapParams p{tile_map, tile_of(cur_c), per_t, (long long)(cslice / kTileElems),
                      tile_of(rimg), per_t, (long long)(rslice / kTileElems), kKtW, status};
      const int kn = (k0 + W < np) ? k0 + W : -1;
      EpiUpdate<W> epi{reinterpret_cast<float*>(A), (size_t)2 * np * np, np, k0, kn, nxt_c, nxt_t, pstride, cslice,
                       tslice};
      epi.red_map = red_map;
      const int slot = instrument ? instr_begin(st) : -1;
      int rc = launch_gemm_persistent<CfgGJH, Split3, 4>(p, 2 * np / CfgGJ::kBn, np / kTileRows, nb, epi, st);
      if (rc) return rc;
      if (instrument) {
        const int live = n - k0 < W ? (n - k0 > 0 ? n - k0 : 0) : W;
        instr_end(slot, st, 8.0 * (double)n * n * live * nb,
                  live > 0 ? 2.0 * sizeof(float2) * (double)n * n * nb : 0.0);
      }
    }
  }
  return NEDMFT_OK;
}

}  // namespace

int gj_blocked_umma(float2* A, int n, int np, int nb, char* scratch, int* status, cudaStream_t st, int width) {
  return gj_width(np, width) == 256 ? gj_blocked_umma_w<256>(A, n, np, nb, scratch, status, st, true)
                             : gj_blocked_umma_w<128>(A, n, np, nb, scratch, status, st, true);
}

// ------------------------------------------------------------------ refinement
//
// One refinement step X1' = X' + X' R' with R' = I - A' X'.  With S split
// into its entries on the pattern of B_q (diagonal, subdiagonal, boundary
// element) and the rest S_d,
//   R'[r] = e_r - [(B - S_sp) X'][i] + [S_d X'][i],   i = row of A behind row r,
// the sparse product is formed exactly (double-float) in the epilogue and the
// dense product S_d X' by an Ozaki split on the bf16 tensor cores: each
// operand is scaled (rows of S_d, columns of X') by a power of two and cut
// into kOzS integer slices of kOzBits bits; every slice product is exact,
// products of equal total slice order d share an FP32 accumulator, and the
// K range is cut into chunks short enough for those integer sums to stay
// exact; the chunk sums are added in double-float.  Only points outside the
// smallest-weight tail (total weight <= kRefineTail) are refined.

namespace {

constexpr int kOzS = 4;           // slices per operand
constexpr int kOzBits = 7;        // bits per slice
constexpr int kOzBn = 64;         // output columns per tile (32 complex)
constexpr int kOzChunkKt = 16;    // K tiles per exact chunk (1024)
constexpr int kRedMaxBatch = 512;
constexpr double kRefineTail = 1e-3;

// double-float helpers (hi + lo, |lo| <= ulp(hi)/2 after renormalisation)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_add(float& h, float& l, float xh, float xl) {
  float s, e;
  two_sum(h, xh, s, e);
  e += l + xl;
  h = s + e;
  l = e - (h - s);
}
// (ch + cl) * x as a double-float
__device__ __forceinline__ void df_mul_f(float ch, float cl, float x, float& h, float& l) {
  const float p = ch * x;
  const float e = fmaf(ch, x, -p);
  h = p;
  l = e + cl * x;
}

struct RefineShared {
  __nv_bfloat16* sd_img;  // kOzS slices of S_d, A operand (np rows, 2np K)
  int* sd_exp;            // per row: exponent of the row scale
  int* flags;             // per point: refine or not
  float2* base;           // -S in FP32, identity padding (np x np)
  size_t sd_slice;
};

// S_d (S without its entries on the pattern of B) -> Ozaki slices, one CTA per row.
__global__ void __launch_bounds__(256) oz_pack_sd_kernel(ContourDev c, const double2* __restrict__ S, int np,
                                                         __nv_bfloat16* __restrict__ img, size_t slice,
                                                         int* __restrict__ exps) {
  const int i = blockIdx.x;
  const int kt = 2 * np / kTileK;
  __shared__ double red[256];
  auto val = [&](int k) -> double2 {
    if (i >= c.n || k >= c.n) return make_double2(0.0, 0.0);
    if (k == i || k == i - 1 || (i == 0 && k == c.n - 1)) return make_double2(0.0, 0.0);
    return S[(size_t)i * c.n + k];
  };
  double m = 0.0;
  for (int k = threadIdx.x; k < np; k += blockDim.x) {
    const double2 z = val(k);
    m = fmax(m, fmax(fabs(z.x), fabs(z.y)));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  int e = 0;
  if (red[0] > 0.0) frexp(red[0], &e);  // red < 2^e
  if (threadIdx.x == 0) exps[i] = e;
  for (int k = threadIdx.x; k < np; k += blockDim.x) {
    const double2 z = val(k);
    double r[2] = {ldexp(z.x, -e), ldexp(z.y, -e)};  // |r| < 1
    for (int sl = 0; sl < kOzS; ++sl) {
      __nv_bfloat16 q[2];
      for (int t = 0; t < 2; ++t) {
        const double v = rint(ldexp(r[t], kOzBits));  // integer, |v| <= 2^kOzBits
        q[t] = __float2bfloat16_rn((float)v);
        r[t] = ldexp(r[t], kOzBits) - v;
      }
      *reinterpret_cast<__nv_bfloat162*>(img + sl * slice + img_offset(i, 2 * k, kt)) = __halves2bfloat162(q[0], q[1]);
    }
  }
}

// flags[q] = 1 unless q lies in the smallest-weight tail of total weight
// <= kRefineTail * sum(w) (weights taken as w_q (1 + |eps| + |ebar|), which
// also bounds the current's quadrature factor).  One CTA; bisection on the
// threshold in log space.
__global__ void __launch_bounds__(1024) refine_select_kernel(const double* __restrict__ eps,
                                                             const double* __restrict__ ebar,
                                                             const double* __restrict__ wq, int nq,
                                                             int* __restrict__ flags) {
  __shared__ double red[1024];
  auto wt = [&](int q) { return fabs(wq[q]) * (1.0 + fabs(eps[q]) + fabs(ebar[q])); };
  auto block_sum = [&](double v) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
  };
  double tot = 0.0;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) tot += wt(q);
  const double total = block_sum(tot);
  double lo = -800.0, hi = 10.0;  // log2 of the threshold
  for (int it = 0; it < 80; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double th = exp2(mid);
    double part = 0.0;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      const double w = wt(q);
      if (w <= th) part += w;
    }
    const double skipped = block_sum(part);
    if (skipped <= kRefineTail * total) lo = mid; else hi = mid;
  }
  const double th = exp2(lo);
  for (int q = threadIdx.x; q < nq; q += blockDim.x) flags[q] = wt(q) > th ? 1 : 0;
}

// Per matrix: the (B - S_sp) coefficients of every row in double-float,
// coef[b][3 i + {0,1,2}] = (diag, sub, boundary) as (re_hi, re_lo, im_hi, im_lo).
__global__ void oz_coef_kernel(ContourDev c, ModelDev m, const double* __restrict__ eps_d,
                               const double* __restrict__ ebar_d, int q0, const double2* __restrict__ S, int np,
                               float4* __restrict__ coef, const int* __restrict__ flags) {
  const int b = blockIdx.y;
  if (!flags[q0 + b]) return;
  const double eps = eps_d[q0 + b], ebar = ebar_d[q0 + b];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    double2 d = make_double2(1.0, 0.0), s = make_double2(0.0, 0.0), k = make_double2(0.0, 0.0);
    if (i < c.n) {
      d = make_double2(-S[(size_t)i * c.n + i].x, 1.0 - S[(size_t)i * c.n + i].y);
      if (i >= 1) s = csub(b_sub(c, m, eps, ebar, i), S[(size_t)i * c.n + i - 1]);
      if (i == 0) k = csub(b_corner(c, m, eps), S[c.n - 1]);
    }
    const double2 v[3] = {d, s, k};
    for (int t = 0; t < 3; ++t) {
      const float rh = (float)v[t].x, ih = (float)v[t].y;
      coef[((size_t)b * np + i) * 3 + t] = make_float4(rh, (float)(v[t].x - rh), ih, (float)(v[t].y - ih));
    }
  }
}

// A'_b = P (B_q - S) in FP32 from the shared base -S (np x np, identity
// padding): row r copies base row i = sigma(r) and adds the three entries of
// B_q in row i.  Block (x, y): rows 32x .. 32x+31 of matrix y; lane r of warp
// 0 forms the B_q entries of row 32x + r (FP64), then warp w copies rows
// w, w + 8, ... with 16-byte loads and stores.
constexpr int kGenRows = 32;
__global__ void __launch_bounds__(256) gen_a_fast_kernel(ContourDev c, ModelDev m, const double* __restrict__ eps_d,
                                                         const double* __restrict__ ebar_d, int q0,
                                                         const float2* __restrict__ base, float2* __restrict__ A,
                                                         int np) {
  const int r0 = blockIdx.x * kGenRows, b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ float2 bv[kGenRows][3];
  __shared__ int bc[kGenRows][3];
  __shared__ int src_row[kGenRows];
  if (warp == 0) {
    const double eps = eps_d[q0 + b], ebar = ebar_d[q0 + b];
    const int r = r0 + lane;
    int i = r;
    if (r < c.n && shifted_point(m, eps)) i = (r + 1 == c.n) ? 0 : r + 1;
    src_row[lane] = i;
    bc[lane][0] = bc[lane][1] = bc[lane][2] = -1;
    if (i < c.n) {
      bc[lane][0] = i;
      bv[lane][0] = make_float2(0.f, 1.f);
      if (i >= 1) {
        const double2 z = b_sub(c, m, eps, ebar, i);
        bc[lane][1] = i - 1;
        bv[lane][1] = make_float2((float)z.x, (float)z.y);
      }
      if (i == 0 && c.n > 1) {
        const double2 z = b_corner(c, m, eps);
        bc[lane][2] = c.n - 1;
        bv[lane][2] = make_float2((float)z.x, (float)z.y);
      }
    }
  }
  __syncthreads();
  for (int rr = warp; rr < kGenRows; rr += 8) {
    const int r = r0 + rr;
    const float4* src = reinterpret_cast<const float4*>(base + (size_t)src_row[rr] * np);
    float4* dst = reinterpret_cast<float4*>(A + (size_t)b * np * np + (size_t)r * np);
    for (int v = lane; v < np / 2; v += 32) {
      float4 x = src[v];
      const int ja = 2 * v, jb = 2 * v + 1;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        if (bc[rr][e] == ja) { x.x += bv[rr][e].x; x.y += bv[rr][e].y; }
        if (bc[rr][e] == jb) { x.z += bv[rr][e].x; x.w += bv[rr][e].y; }
      }
      dst[v] = x;
    }
  }
}

__global__ void base_neg_s_kernel(ContourDev c, const double2* __restrict__ S, float2* __restrict__ base, int np) {
  const int r = blockIdx.x;
  for (int j = threadIdx.x; j < np; j += blockDim.x) {
    float2 v;
    if (r < c.n && j < c.n) { const double2 z = S[(size_t)r * c.n + j]; v = make_float2((float)-z.x, (float)-z.y); }
    else v = make_float2(r == j ? 1.f : 0.f, 0.f);
    base[(size_t)r * np + j] = v;
  }
}

// Per refined matrix: Ozaki slices of X' as the residual's B operand (rows
// n = 2j, 2j+1; k = 2k', 2k'+1; [[re, -im], [im, re]] of X'[k'][j]) with a
// power-of-two scale per column j, and X' hi/lo as the correction's A
// operand.  Block (x, y): complex columns x*32 .. +31 of matrix y; tiles of
// 32 x 32 pass through shared memory, and both images are written in whole
// 16-byte core-matrix rows.
__global__ void __launch_bounds__(256) oz_pack_x_kernel(const float2* __restrict__ X, int np, int q0,
                                                        const int* __restrict__ flags, __nv_bfloat16* __restrict__ ximg,
                                                        int* __restrict__ xexp, __nv_bfloat16* __restrict__ aimg) {
  const int b = blockIdx.y;
  if (!flags[q0 + b]) return;
  const int j0 = blockIdx.x * 32;
  const float2* x = X + (size_t)b * np * np;
  const int kt = 2 * np / kTileK;
  const size_t xs = (size_t)2 * np * 2 * np, as = (size_t)np * 2 * np;
  __nv_bfloat16* xi = ximg + b * kOzS * xs;
  __nv_bfloat16* ai = aimg + b * 2 * as;
  __shared__ float colmax[8][32];
  __shared__ int cexp[32];
  __shared__ float2 tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  float m = 0.f;
  for (int k = ty; k < np; k += 8) {
    const float2 z = x[(size_t)k * np + j0 + tx];
    m = fmaxf(m, fmaxf(fabsf(z.x), fabsf(z.y)));
  }
  colmax[ty][tx] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    float mm = 0.f;
    for (int g = 0; g < 8; ++g) mm = fmaxf(mm, colmax[g][threadIdx.x]);
    int e = 0;
    if (mm > 0.f) frexpf(mm, &e);
    cexp[threadIdx.x] = e;
    xexp[(size_t)b * np + j0 + threadIdx.x] = e;
  }
  __syncthreads();
  for (int k0 = 0; k0 < np; k0 += 32) {
    // coalesced load of rows k0 .. k0+31, columns j0 .. j0+31
    for (int rr = ty; rr < 32; rr += 8) tile[rr][tx] = x[(size_t)(k0 + rr) * np + j0 + tx];
    __syncthreads();
    {
      // the A image (hi, lo): thread t writes one 16-byte core-matrix row,
      // row k = k0 + 8 (t / 64) + t % 8 and entries j0 + 4 c .. +3, c = (t / 8) % 8,
      // so 8 consecutive threads fill one 128-byte core matrix
      const int t = threadIdx.x;
      const int kr = 8 * (t >> 6) + (t & 7), c = (t >> 3) & 7;
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 z = tile[kr][4 * c + q];
        __nv_bfloat16 rh, rl, ih, il;
        split2(z.x, rh, rl);
        split2(z.y, ih, il);
        hi[q] = bf2_bits(rh, ih);
        lo[q] = bf2_bits(rl, il);
      }
      const size_t o = img_offset(k0 + kr, 2 * (j0 + 4 * c), kt);
      *reinterpret_cast<uint4*>(ai + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(ai + as + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    {
      // the B image: rows 2j, 2j+1 (j = j0 + 4 g + p, g = t / 32, p = t % 4) and
      // k = k0 + 4 c .. +3 (c = (t / 4) % 8): two 16-byte core-matrix rows per
      // slice, 4 consecutive threads fill one core matrix
      const int t = threadIdx.x;
      const int jl = 4 * (t >> 5) + (t & 3), c = (t >> 2) & 7;
      const int j = j0 + jl;
      const int e = cexp[jl];
      float r[4][2];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 z = tile[4 * c + q][jl];
        r[q][0] = ldexpf(z.x, -e);
        r[q][1] = ldexpf(z.y, -e);
      }
      const size_t o0 = img_offset(2 * j, 2 * (k0 + 4 * c), kt), o1 = img_offset(2 * j + 1, 2 * (k0 + 4 * c), kt);
      for (int sl = 0; sl < kOzS; ++sl) {
        uint32_t ev[4], od[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float qv[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            qv[u] = rintf(ldexpf(r[q][u], kOzBits));
            r[q][u] = ldexpf(r[q][u], kOzBits) - qv[u];
          }
          const __nv_bfloat16 re = __float2bfloat16_rn(qv[0]), im = __float2bfloat16_rn(qv[1]);
          const __nv_bfloat16 nim = __float2bfloat16_rn(-qv[1]);
          ev[q] = bf2_bits(re, nim);  // row 2j: [re, -im]
          od[q] = bf2_bits(im, re);   // row 2j+1: [im, re]
        }
        *reinterpret_cast<uint4*>(xi + sl * xs + o0) = make_uint4(ev[0], ev[1], ev[2], ev[3]);
        *reinterpret_cast<uint4*>(xi + sl * xs + o1) = make_uint4(od[0], od[1], od[2], od[3]);
      }
    }
    __syncthreads();
  }
}

struct OzParams {
  CUtensorMap a_map;       // S_d slices (shared), packed tiles from the first slice
  CUtensorMap b_map;       // X' slices of the batch, packed tiles from matrix 0
  long long a_slice;       // tiles between S_d slices
  long long b_batch, b_slice;  // tiles between matrices / slices of X'
  const int* a_exp;        // row exponents
  const int* b_exp;        // column exponents per matrix (np each)
  const float2* X;         // X' per matrix (np x np)
  const float4* coef;      // per matrix (np x 3)
  const int* flags;
  __nv_bfloat16* rimg;     // R' as the correction's B operand, hi/lo
  size_t r_batch, r_slice;
  ContourDev c;
  ModelDev m;
  const double* eps;
  int q0, nb, np, kt;
  int* status;
};

// Stages of half tiles (32 k): A kOzS x 8 KB, B (64 rows) kOzS x 4 KB.
constexpr int kOzHalfA = kTileBytes / 2, kOzHalfB = kTileBytes / 4;
constexpr int kOzStageBytes = kOzS * (kOzHalfA + kOzHalfB);  // 48 KB
constexpr int kOzStages = 4;
constexpr int kOzEpiW = 8;                     // epilogue warps: two per TMEM lane quarter
constexpr int kOzEpiCols = kOzBn * 4 / kOzEpiW;  // accumulator columns per epilogue thread
constexpr int kOzSmem = kOzStages * kOzStageBytes + 1024 + 256;

// Persistent: the units (refined matrix, m tile, n tile), m fastest, are
// dealt round-robin to the CTAs.  Consecutive units share the B tile and all
// share A (S_d), which stays in L2.  Chunks of kOzChunkKt K tiles alternate
// between two TMEM buffers of kOzS accumulators of kOzBn columns across units,
// so the epilogue drains (and finishes a unit) while the next chunk is
// multiplied.
struct OzBars {
  uint64_t full[kOzStages], empty[kOzStages], acc_full[2], acc_empty[2], drain;
  uint32_t tmem_slot;
  int abort;
};
static_assert(sizeof(OzBars) <= 256, "residual barrier block");

__global__ void __launch_bounds__(64 + 32 * kOzEpiW, 1) oz_residual_kernel(const __grid_constant__ OzParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  OzBars& bars = *reinterpret_cast<OzBars*>(smem + kOzStages * kOzStageBytes);
  uint64_t* full = bars.full;
  uint64_t* empty = bars.empty;
  uint64_t* acc_full = bars.acc_full;
  uint64_t* acc_empty = bars.acc_empty;
  volatile int* abort_flag = &bars.abort;
  __shared__ int refined[kRedMaxBatch];
  __shared__ int n_refined;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_tiles = p.np / kTileRows, n_tiles = 2 * p.np / kOzBn;
  const int per = m_tiles * n_tiles;
  const int kh = 2 * p.kt;                  // half tiles per unit
  const int hc = 2 * kOzChunkKt;            // half tiles per chunk
  const int nchunks = (kh + hc - 1) / hc;   // chunks per unit

  if (threadIdx.x == 0) {
    for (int s = 0; s < kOzStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&acc_full[s], 1);
      mbar_init(&acc_empty[s], 32 * kOzEpiW);
    }
    mbar_init(&bars.drain, 1);
    *abort_flag = 0;
    fence_barrier_init();
    int r = 0;
    for (int b = 0; b < p.nb; ++b)
      if (p.flags[p.q0 + b]) refined[r++] = b;
    n_refined = r;
  }
  if (warp == 1) tmem_alloc(&bars.tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars.tmem_slot;
  const int units = n_refined * per;
  const int G = gridDim.x, cl = blockIdx.x;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int u = cl; u < units && ok; u += G) {
        const int bidx = refined[u / per], rem = u % per;
        const int mt = rem % m_tiles, nt = rem / m_tiles;
        const long long a0 = (long long)mt * p.kt;
        // B rows nt * 64 .. +63: row groups 8 (nt & 1) .. +7 of tile nt / 2
        const long long b0 = bidx * p.b_batch + (long long)(nt >> 1) * p.kt;
        const int rg = 8 * (nt & 1);
        for (int h = 0; h < kh; ++h, ++it) {
          const int s = it % kOzStages;
          const uint32_t ph = (it / kOzStages) & 1;
          if (!mbar_wait(&empty[s], ph ^ 1, abort_flag)) { ok = false; break; }
          unsigned char* st = smem + s * kOzStageBytes;
          const int kt = h >> 1, kc = 4 * (h & 1);
          mbar_arrive_expect_tx(&full[s], kOzStageBytes);
          for (int sl = 0; sl < kOzS; ++sl)
            tma_load_4d(&p.a_map, st + sl * kOzHalfA, 0, kc, 0, (int)(a0 + sl * p.a_slice + kt), &full[s]);
          for (int sl = 0; sl < kOzS; ++sl)
            tma_load_4d(&p.b_map, st + kOzS * kOzHalfA + sl * kOzHalfB, 0, kc, rg, (int)(b0 + sl * p.b_slice + kt),
                        &full[s]);
        }
      }
      // no copy may be left in flight at exit
      for (int k = it - kOzStages < 0 ? 0 : it - kOzStages; k < it; ++k) {
        const uint64_t t0 = global_ns();
        while (!mbar_test(&full[k % kOzStages], (k / kOzStages) & 1) && global_ns() - t0 < kDrainNs) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      int it = 0, cg = 0;  // stage uses, chunks (across units)
      for (int u = cl; u < units && ok; u += G) {
        for (int h = 0; h < kh && ok; ++h, ++it) {
          const bool first = (h % hc) == 0;
          const int buf = cg & 1;
          if (first && cg >= 2) {
            if (!mbar_wait(&acc_empty[buf], ((cg >> 1) - 1) & 1, abort_flag)) { ok = false; break; }
            tc_fence_after();
          }
          const int s = it % kOzStages;
          if (!mbar_wait(&full[s], (it / kOzStages) & 1, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + s * kOzStageBytes);
          // The B slices lie back to back (64 rows each, 8-row groups 512 B
          // apart), so B_0 .. B_{kOzS-1-a} form one operand of (kOzS - a) * 64
          // rows: one MMA per A slice a writes A_a B_b to accumulator
          // d = a + b (columns d * kOzBn), and a = 0 opens every order.
#pragma unroll
          for (int kk = 0; kk < kTileK / 32; ++kk) {
            const uint32_t b_addr = st + kOzS * kOzHalfA + kk * 256;
#pragma unroll
            for (int a = 0; a < kOzS; ++a) {
              const uint32_t a_addr = st + a * kOzHalfA + kk * 256;
              mma_bf16(tmem + buf * 256 + a * kOzBn, smem_desc(a_addr, 128, 512), smem_desc(b_addr, 128, 512),
                       idesc_bf16(128, (kOzS - a) * kOzBn), (first && kk == 0 && a == 0) ? 0u : 1u);
            }
          }
          mma_commit(&empty[s]);
          if ((h % hc) == hc - 1 || h == kh - 1) {
            mma_commit(&acc_full[buf]);
            ++cg;
          }
        }
      }
      // completes when every product issued above has (also after an abort)
      mma_commit(&bars.drain);
    }
  } else {
    // kOzEpiW epilogue warps: warp w owns TMEM lanes 32 (w % 4) .. +31 (rows of
    // the tile) and columns kOzEpiCols (w - 2) / 4 .. + kOzEpiCols - 1 of each order
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const int part = (warp - 2) >> 2;
    bool ok = true;
    int cg = 0;
    for (int u = cl; u < units && ok; u += G) {
      const int bidx = refined[u / per], rem = u % per;
      const int mt = rem % m_tiles, nt = rem / m_tiles;
      const int i = mt * kTileRows + row;  // output row of S_d X'
      const int n = p.c.n, np = p.np;
      const bool sh = shifted_point(p.m, p.eps[p.q0 + bidx]);
      const int r = (i < n && sh) ? (i == 0 ? n - 1 : i - 1) : i;  // row of R' fed by row i
      const int ei = p.a_exp[i];
      const int* xe = p.b_exp + (size_t)bidx * np;
      const int j0 = nt * (kOzBn / 2) + part * (kOzEpiCols / 2);  // this thread's first complex column
      // The sums start from T - (B - S_sp) X' at (i, j) (double-float, in the
      // accumulator's units 2^(e_i + e_j)), so the reads of X' rows (16-byte
      // vectors) overlap the products of the unit's first chunk.
      float hs[kOzEpiCols], ls[kOzEpiCols];
      {
        const float2* x = p.X + (size_t)bidx * np * np;
        const float4* cf = p.coef + (size_t)bidx * np * 3;
        // the diagonal, and one off-diagonal entry: the subdiagonal (row i - 1)
        // for 1 <= i < n, the corner (row n - 1) for i = 0, none beyond n
        const float4 cd = cf[3 * i], co = i == 0 ? cf[2] : cf[3 * i + 1];
        const float4* xd = reinterpret_cast<const float4*>(x + (size_t)i * np + j0);
        const int io = i == 0 ? n - 1 : i - 1;
        const float4* xo = i < n ? reinterpret_cast<const float4*>(x + (size_t)io * np + j0) : nullptr;
#pragma unroll
        for (int v = 0; v < kOzEpiCols / 4; ++v) {  // two complex columns per vector
          const float4 zd = xd[v];
          const float4 zo = xo ? xo[v] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int uu = 2 * v + h, j = j0 + uu;
            float tr_h = 0.f, tr_l = 0.f, ti_h = 0.f, ti_l = 0.f;
            auto sub_prod = [&](float4 co, float xr, float xi) {
              float hh, ll;
              df_mul_f(co.x, co.y, xr, hh, ll); df_add(tr_h, tr_l, -hh, -ll);  // - c_re x_re
              df_mul_f(co.z, co.w, xi, hh, ll); df_add(tr_h, tr_l, hh, ll);    // + c_im x_im
              df_mul_f(co.x, co.y, xi, hh, ll); df_add(ti_h, ti_l, -hh, -ll);  // - c_re x_im
              df_mul_f(co.z, co.w, xr, hh, ll); df_add(ti_h, ti_l, -hh, -ll);  // - c_im x_re
            };
            sub_prod(cd, h ? zd.z : zd.x, h ? zd.w : zd.y);
            if (xo) sub_prod(co, h ? zo.z : zo.x, h ? zo.w : zo.y);
            if (r == j) df_add(tr_h, tr_l, 1.0f, 0.0f);
            const int sc = -(ei + xe[j]);
            hs[2 * uu] = ldexpf(tr_h, sc);
            ls[2 * uu] = ldexpf(tr_l, sc);
            hs[2 * uu + 1] = ldexpf(ti_h, sc);
            ls[2 * uu + 1] = ldexpf(ti_l, sc);
          }
        }
      }
      for (int ch = 0; ch < nchunks; ++ch, ++cg) {
        const int buf = cg & 1;
        if (!mbar_wait(&acc_full[buf], (cg >> 1) & 1, abort_flag)) { ok = false; break; }
        tc_fence_after();
#pragma unroll
        for (int d = 0; d < kOzS; ++d) {
          const float sc = ldexpf(1.0f, -kOzBits * (d + 2));
#pragma unroll
          for (int pc = 0; pc < kOzEpiCols / 32; ++pc) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + buf * 256 + d * kOzBn + part * kOzEpiCols + pc * 32, v);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              float s, er;
              two_sum(hs[pc * 32 + e], v[e] * sc, s, er);
              hs[pc * 32 + e] = s;
              ls[pc * 32 + e] += er;
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&acc_empty[buf]);
      }
      if (!ok || *abort_flag) break;
      __nv_bfloat16* ri = p.rimg + bidx * p.r_batch;
      const int kt = 2 * np / kTileK;
#pragma unroll
      for (int uu = 0; uu < kOzEpiCols / 2; ++uu) {
        const int j = j0 + uu;
        const int sc = ei + xe[j];
        const float tr_h = ldexpf(hs[2 * uu], sc), tr_l = ldexpf(ls[2 * uu], sc);
        const float ti_h = ldexpf(hs[2 * uu + 1], sc), ti_l = ldexpf(ls[2 * uu + 1], sc);
        const float re = tr_h + tr_l, im = ti_h + ti_l;
        __nv_bfloat16 rh, rl, ih, il, nh, nl;
        split2(re, rh, rl);
        split2(im, ih, il);
        split2(-im, nh, nl);
        const size_t o0 = img_offset(2 * j, 2 * r, kt), o1 = img_offset(2 * j + 1, 2 * r, kt);
        *reinterpret_cast<__nv_bfloat162*>(ri + o0) = __halves2bfloat162(rh, nh);
        *reinterpret_cast<__nv_bfloat162*>(ri + o1) = __halves2bfloat162(ih, rh);
        *reinterpret_cast<__nv_bfloat162*>(ri + p.r_slice + o0) = __halves2bfloat162(rl, nl);
        *reinterpret_cast<__nv_bfloat162*>(ri + p.r_slice + o1) = __halves2bfloat162(il, rl);
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    // the tensor core must be idle before the columns are released
    const uint64_t t0 = global_ns();
    while (!mbar_test(&bars.drain, 0) && global_ns() - t0 < kDrainNs) {
    }
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && *abort_flag && p.status) atomicCAS(p.status, 0, DS_TIMEOUT);
}

// dX' = acc (FP32 interleaved).
// and its bf16 image as the A operand of the second-order term dX' R' (row i,
// k = 2j, 2j+1: the 32 values of a chunk are 32 consecutive k, four 16-byte
// core-matrix rows).
struct EpiStore {
  float* out;
  size_t bstride;  // floats between matrices
  int np;
  __nv_bfloat16* img;
  size_t img_stride;  // elements between matrices
  __device__ void operator()(int b, int mt, int nt, int r, int c0, const float* v) const {
    const int i = mt * kTileRows + r;
    const int k0 = nt * CfgGJ::kBn + c0;
    float* row = out + b * bstride + (size_t)i * 2 * np + k0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      *reinterpret_cast<float4*>(row + 4 * u) = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
    __nv_bfloat16* im = img + b * img_stride;
    const int kt = 2 * np / kTileK;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      uint32_t h[4];
#pragma unroll
      for (int e = 0; e < 4; ++e)
        h[e] = bf2_bits(__float2bfloat16_rn(v[8 * g + 2 * e]), __float2bfloat16_rn(v[8 * g + 2 * e + 1]));
      *reinterpret_cast<uint4*>(im + img_offset(i, k0 + 8 * g, kt)) = make_uint4(h[0], h[1], h[2], h[3]);
    }
  }
};

// dX' += acc (FP32 interleaved): the second-order term of the refinement.
struct EpiAdd {
  float* out;
  size_t bstride;  // floats between matrices
  int np;
  __device__ void operator()(int b, int mt, int nt, int r, int c0, const float* v) const {
    const int i = mt * kTileRows + r;
    float4* row = reinterpret_cast<float4*>(out + b * bstride + (size_t)i * 2 * np + nt * CfgGJ::kBn + c0);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      float4 x = row[u];
      x.x += v[4 * u]; x.y += v[4 * u + 1]; x.z += v[4 * u + 2]; x.w += v[4 * u + 3];
      row[u] = x;
    }
  }
};

// gloc (= or +=) sum_b wq (X' + flag dX')[i][col(j)], b ascending.  The sum
// runs in double-float (hi + lo FP32 pairs); w_q is split into hi + lo and
// X' is exact in FP32, so w_q X' is formed exactly (two-product).
__global__ void __launch_bounds__(256) reduce_refined_kernel(ContourDev c, ModelDev m,
                                                             const double* __restrict__ eps_d,
                                                             const double* __restrict__ wq_d, int q0, int nb,
                                                             const float2* __restrict__ X,
                                                             const float2* __restrict__ dX,
                                                             const int* __restrict__ flags, int np, bool first,
                                                             double2* __restrict__ gloc) {
  __shared__ float wh[kRedMaxBatch], wl[kRedMaxBatch];
  __shared__ unsigned char shf[kRedMaxBatch], rf[kRedMaxBatch];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double w = wq_d[q0 + b];
    wh[b] = (float)w;
    wl[b] = (float)(w - (double)wh[b]);
    shf[b] = shifted_point(m, eps_d[q0 + b]) ? 1 : 0;
    rf[b] = flags[q0 + b] ? 1 : 0;
  }
  __syncthreads();
  const size_t total = (size_t)c.n * c.n, mat = (size_t)np * np;
  // entries e = i n + j dealt evenly to all threads (consecutive threads, consecutive j)
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    {
      const int i = (int)(e / c.n), j = (int)(e - (size_t)i * c.n);
      float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
      const int j0 = j, j1 = (j == 0 ? c.n - 1 : j - 1);
      // eight matrices' loads in flight at a time; the sum still runs over b in order
      constexpr int U = 8;
      for (int b0 = 0; b0 < nb; b0 += U) {
        float2 xs[U], ds[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int b = b0 + u;
          xs[u] = make_float2(0.f, 0.f);
          ds[u] = make_float2(0.f, 0.f);
          if (b < nb) {
            const size_t off = b * mat + (size_t)i * np + (shf[b] ? j1 : j0);
            xs[u] = X[off];
            if (rf[b]) ds[u] = dX[off];
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int b = b0 + u;
          if (b >= nb) break;
          const float2 x = xs[u];
          const float h = wh[b], l = wl[b];
          float px = h * x.x, ex = fmaf(h, x.x, -px) + l * x.x;
          float py = h * x.y, ey = fmaf(h, x.y, -py) + l * x.y;
          if (rf[b]) {
            ex += h * ds[u].x;
            ey += h * ds[u].y;
          }
          df_add(rh, rl, px, ex);
          df_add(ih, il, py, ey);
        }
      }
      double2 acc = first ? make_double2(0.0, 0.0) : gloc[e];
      acc.x += (double)rh + (double)rl;
      acc.y += (double)ih + (double)il;
      gloc[e] = acc;
    }
  }
}

// One warp per time t_m: lane l takes the points b = l, l + 32, ... of the
// batch, and the lanes' partial sums are added in a fixed shuffle tree.
__global__ void __launch_bounds__(256) reduce_refined_current_kernel(
    ContourDev c, ModelDev mo, const double* __restrict__ eps_d, const double* __restrict__ ebar_d,
    const double* __restrict__ wq_d, int q0, int nb, const float2* __restrict__ X, const float2* __restrict__ dX,
    const int* __restrict__ flags, int np, bool first, double2* __restrict__ jacc) {
  const int mm = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (mm >= c.nt) return;  // whole warps
  const double t = t_re(c, mm);
  const int jcol = 2 * c.nt - mm;
  const size_t mat = (size_t)np * np;
  // ebar_q(t) = ebar cos(Et) + eps sin(Et) for t > 0 (ebar before): the
  // trigonometric factors are the same for every point
  double sn = 0.0, cs = 1.0;
  if (t > 0.0) sincos(mo.E * t, &sn, &cs);
  double2 part = make_double2(0.0, 0.0);
#pragma unroll 4
  for (int b = lane; b < nb; b += 32) {
    const int q = q0 + b;
    const size_t off = b * mat + (size_t)mm * np + unshift_col(jcol, c.n, shifted_point(mo, eps_d[q]));
    double2 v = to_d(X[off]);
    if (flags[q]) v = cadd(v, to_d(dX[off]));
    const double w = wq_d[q] * (ebar_d[q] * cs + eps_d[q] * sn);
    part.x = fma(w, v.x, part.x);
    part.y = fma(w, v.y, part.y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    part.x += __shfl_xor_sync(0xffffffffu, part.x, o);
    part.y += __shfl_xor_sync(0xffffffffu, part.y, o);
  }
  if (lane == 0) {
    double2 acc = first ? make_double2(0.0, 0.0) : jacc[mm];
    acc.x += part.x;
    acc.y += part.y;
    jacc[mm] = acc;
  }
}

// Refinement buffers, each an array over the batch.
struct RefineLayout {
  size_t ximg, xexp, aimg, rimg, coef, dx, total;  // bytes per region
};
RefineLayout refine_layout(int np, int nb) {
  RefineLayout r{};
  r.ximg = align1k(kOzS * sizeof(__nv_bfloat16) * (size_t)2 * np * 2 * np * nb);
  r.xexp = align1k(sizeof(int) * (size_t)np * nb);
  r.aimg = align1k(2 * sizeof(__nv_bfloat16) * (size_t)np * 2 * np * nb);
  r.rimg = align1k(2 * sizeof(__nv_bfloat16) * (size_t)2 * np * 2 * np * nb);
  r.coef = align1k(sizeof(float4) * (size_t)np * 3 * nb);
  r.dx = align1k(sizeof(float2) * (size_t)np * np * nb);
  r.total = r.ximg + r.xexp + r.aimg + r.rimg + r.coef + r.dx;
  return r;
}

RefineShared shared_layout(char* shared, int np, int nq) {
  RefineShared r{};
  r.sd_slice = (size_t)np * 2 * np;
  r.sd_img = reinterpret_cast<__nv_bfloat16*>(shared);
  r.sd_exp = reinterpret_cast<int*>(shared + align1k(kOzS * sizeof(__nv_bfloat16) * r.sd_slice));
  r.flags = reinterpret_cast<int*>(reinterpret_cast<char*>(r.sd_exp) + align1k(sizeof(int) * (size_t)np));
  r.base = reinterpret_cast<float2*>(reinterpret_cast<char*>(r.flags) + align1k(sizeof(int) * (size_t)nq));
  return r;
}
size_t flags_bytes(int nq) { return align1k(sizeof(int) * (size_t)nq); }

}  // namespace

// ------------------------------------------------------------------ lattice batch on this path

int umma_block_width(int np, int width) { return gj_width(np, width); }
int umma_padded(int n, int width) {
  const int p128 = ((n + 127) / 128) * 128, p256 = ((n + 255) / 256) * 256;
  if (n <= 512 || width == 128) return p128;
  if (width == 256) return p256;
  // the default: 128-column steps read and write the matrix twice as often
  // (measured ~1.2x the time per flop at N_c = 1000 - 1500), so they pay only
  // where padding to 128 instead of 256 saves more than a fifth of the flops
  // (N_c = 1300: 1408 vs 1536 rows, 209 vs 227 ms per lattice step)
  const double r = (double)p128 / p256;
  return (p128 < p256 && r * r * r < 0.8) ? p128 : p256;
}
size_t umma_batch_bytes_per_matrix(int np, int width) {
  return gj_buffers_for(np, width).total + refine_layout(np, 1).total;
}
int umma_default_batch(int np) { return np <= 2048 ? 152 : 76; }
size_t umma_shared_bytes(int np, int nq) {
  return align1k(kOzS * sizeof(__nv_bfloat16) * (size_t)np * 2 * np) + align1k(sizeof(int) * (size_t)np) +
         flags_bytes(nq) + align1k(sizeof(float2) * (size_t)np * np);
}
size_t umma_batch_bytes(int np, int nb, int width) {
  return gj_buffers_for(np, width).total * nb + refine_layout(np, nb).total;
}

int umma_prepare_shared(const ContourDev& c, const double2* S, int np, const double* eps, const double* ebar,
                        const double* wq, int nq, char* shared, cudaStream_t st) {
  RefineShared r = shared_layout(shared, np, nq);
  base_neg_s_kernel<<<np, 256, 0, st>>>(c, S, r.base, np);
  NED_LAUNCH_CHECK("base_neg_s_kernel");
  oz_pack_sd_kernel<<<np, 256, 0, st>>>(c, S, np, r.sd_img, r.sd_slice, r.sd_exp);
  NED_LAUNCH_CHECK("oz_pack_sd_kernel");
  refine_select_kernel<<<1, 1024, 0, st>>>(eps, ebar, wq, nq, r.flags);
  NED_LAUNCH_CHECK("refine_select_kernel");
  return NEDMFT_OK;
}

namespace {
// 4-D tensor map over `tiles` packed 128 x 64 bf16 tiles at `base`, moved in
// half tiles of `rgroups` 8-row groups: box (64 elements, 4 core columns, rgroups, 1).
int encode_oz_map(CUtensorMap* map, void* base, uint64_t tiles, uint32_t rgroups) {
  const EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return set_error(NEDMFT_ECUDA, "cuTensorMapEncodeTiled is not available from the CUDA driver");
  const cuuint64_t dims[4] = {64, 8, 16, tiles};
  const cuuint64_t strides[3] = {128, 1024, 16384};
  const cuuint32_t box[4] = {64, 4, rgroups, 1};
  const cuuint32_t elem_strides[4] = {1, 1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, elem_strides,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(NEDMFT_ECUDA, "cuTensorMapEncodeTiled (residual) failed (CUresult %d)", (int)r);
  return NEDMFT_OK;
}
}  // namespace

int umma_lattice_batch(const ContourDev& c, const ModelDev& m, const double* eps, const double* ebar,
                       const double* wq, int q0, int nb, int nq_total, int np, const double2* S, char* shared,
                       char* batch, bool first, double2* gloc, double2* jacc, int* status, cudaStream_t st,
                       int width) {
  const GjBuffers g = gj_buffers_for(np, width);
  const RefineShared sh = shared_layout(shared, np, nq_total);
  const int mb_alloc = nb;  // regions are sized for this batch by the caller's layout
  (void)mb_alloc;
  // layout: nb matrices | nb GJ panel scratch | refinement regions
  float2* X = reinterpret_cast<float2*>(batch);
  char* scratch = batch + g.mat * nb;
  const RefineLayout rl = refine_layout(np, nb);
  char* rbase = scratch + g.scratch * nb;
  __nv_bfloat16* ximg = reinterpret_cast<__nv_bfloat16*>(rbase);
  int* xexp = reinterpret_cast<int*>(rbase + rl.ximg);
  __nv_bfloat16* aimg = reinterpret_cast<__nv_bfloat16*>(rbase + rl.ximg + rl.xexp);
  __nv_bfloat16* rimg = reinterpret_cast<__nv_bfloat16*>(rbase + rl.ximg + rl.xexp + rl.aimg);
  float4* coef = reinterpret_cast<float4*>(rbase + rl.ximg + rl.xexp + rl.aimg + rl.rimg);
  float2* dx = reinterpret_cast<float2*>(rbase + rl.ximg + rl.xexp + rl.aimg + rl.rimg + rl.coef);
  const size_t mat = (size_t)np * np;
  const size_t xs = (size_t)2 * np * 2 * np, as = (size_t)np * 2 * np, rs = (size_t)2 * np * 2 * np;
  int rc;
  gen_a_fast_kernel<<<dim3(np / kGenRows, nb), 256, 0, st>>>(c, m, eps, ebar, q0, sh.base, X, np);
  NED_LAUNCH_CHECK("gen_a_fast_kernel");
  if ((rc = gj_blocked_umma(X, c.n, np, nb, scratch, status, st, width))) return rc;
  oz_coef_kernel<<<dim3((np + 255) / 256, nb), 256, 0, st>>>(c, m, eps, ebar, q0, S, np, coef, sh.flags);
  NED_LAUNCH_CHECK("oz_coef_kernel");
  oz_pack_x_kernel<<<dim3(np / 32, nb), 256, 0, st>>>(X, np, q0, sh.flags, ximg, xexp, aimg);
  NED_LAUNCH_CHECK("oz_pack_x_kernel");
  {
    OzParams p{};
    const uint64_t xs_tiles = (uint64_t)xs / kTileElems;  // tiles per X' slice
    if ((rc = encode_oz_map(&p.a_map, sh.sd_img, (uint64_t)kOzS * sh.sd_slice / kTileElems, 16))) return rc;
    if ((rc = encode_oz_map(&p.b_map, ximg, (uint64_t)nb * kOzS * xs_tiles, 8))) return rc;
    p.a_slice = (long long)(sh.sd_slice / kTileElems);
    p.b_batch = (long long)(kOzS * xs_tiles);
    p.b_slice = (long long)xs_tiles;
    p.a_exp = sh.sd_exp;
    p.b_exp = xexp;
    p.X = X; p.coef = coef; p.flags = sh.flags;
    p.rimg = rimg; p.r_batch = 2 * rs; p.r_slice = rs;
    p.c = c; p.m = m; p.eps = eps; p.q0 = q0; p.nb = nb; p.np = np; p.kt = 2 * np / kTileK; p.status = status;
    if (nb > kRedMaxBatch) return set_error(NEDMFT_EINVAL, "residual: batch %d > %d", nb, kRedMaxBatch);
    // one CTA per SM, persistent over the refined matrices' units
    int sms = 0;
    if ((rc = ensure_dyn_smem(reinterpret_cast<const void*>(oz_residual_kernel), kOzSmem))) return rc;
    if ((rc = device_sm_count(&sms))) return rc;
    oz_residual_kernel<<<sms, 64 + 32 * kOzEpiW, kOzSmem, st>>>(p);
    NED_LAUNCH_CHECK("oz_residual_kernel");
  }
  // dX' = X' R' + (X' R') R' (refined points only): the first two terms of
  // X' (I - R')^-1 - X' = X' (R' + R'^2 + ...), both with the one residual R'.
  // The first product in bf16x3; the second, |R'| times smaller, as one bf16
  // product from the bf16 image of X' R' that the first one's epilogue writes
  // (into the X' slice buffer, which the residual no longer needs).
  {
    GemmParams p{aimg, 2 * as, as, rimg, 2 * rs, rs, 2 * np / kTileK, status};
    EpiStore epi{reinterpret_cast<float*>(dx), 2 * mat, np, ximg, kOzS * xs};
    if ((rc = ensure_dyn_smem(reinterpret_cast<const void*>(umma_gemm_flag_kernel<CfgGJ, Split3, EpiStore>),
                              CfgGJ::kSmem)))
      return rc;
    umma_gemm_flag_kernel<CfgGJ, Split3, EpiStore>
        <<<dim3(2 * np / CfgGJ::kBn, np / kTileRows, nb), 192, CfgGJ::kSmem, st>>>(p, epi, sh.flags, q0);
    NED_LAUNCH_CHECK("umma_gemm_flag_kernel");
  }
  {
    GemmParams p{ximg, kOzS * xs, 0, rimg, 2 * rs, rs, 2 * np / kTileK, status};
    EpiAdd epi{reinterpret_cast<float*>(dx), 2 * mat, np};
    if ((rc = ensure_dyn_smem(reinterpret_cast<const void*>(umma_gemm_flag_kernel<CfgHi, Split1, EpiAdd>),
                              CfgHi::kSmem)))
      return rc;
    umma_gemm_flag_kernel<CfgHi, Split1, EpiAdd>
        <<<dim3(2 * np / CfgHi::kBn, np / kTileRows, nb), 192, CfgHi::kSmem, st>>>(p, epi, sh.flags, q0);
    NED_LAUNCH_CHECK("umma_gemm_flag_kernel");
  }
  {
    // as many rounds of 152 x 8 blocks as the entries need, then just enough
    // blocks for that many rounds, so every thread takes the same count
    const size_t total = (size_t)c.n * c.n, wave = (size_t)152 * 8 * 256;
    const size_t rounds = total > wave ? (total + wave - 1) / wave : 1;
    const int bx = total ? (int)((total + rounds * 256 - 1) / (rounds * 256)) : 1;
    if (nb > kRedMaxBatch) return set_error(NEDMFT_EINVAL, "reduce: batch %d > %d", nb, kRedMaxBatch);
    reduce_refined_kernel<<<bx, 256, 0, st>>>(c, m, eps, wq, q0, nb, X, dx, sh.flags, np, first, gloc);
    NED_LAUNCH_CHECK("reduce_refined_kernel");
    if (jacc) {
      reduce_refined_current_kernel<<<ceil_div(c.nt, 8), 256, 0, st>>>(c, m, eps, ebar, wq, q0, nb, X, dx,
                                                                         sh.flags, np, first, jacc);
      NED_LAUNCH_CHECK("reduce_refined_current_kernel");
    }
  }
  return NEDMFT_OK;
}

namespace {
// One CTA waits (bounded) on an mbarrier that nothing arrives at: the wait
// runs out after the device's wait limit and records DS_TIMEOUT.
__global__ void wait_selftest_kernel(int* status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  abort_flag = 0;
  fence_barrier_init();
  if (!mbar_wait(&bar, 0, &abort_flag) && status) atomicCAS(status, 0, DS_TIMEOUT);
}
}  // namespace

int umma_wait_selftest(int* status, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(status);
  NED_LAUNCH_CHECK("wait_selftest_kernel");
  return NEDMFT_OK;
}

// Limit of the bounded waits of the tensor-core kernels on the current device
// (this file's and the impurity update's; stream-ordered after earlier work
// on `st`).
int umma_set_wait_ns(uint64_t ns, cudaStream_t st) {
  NED_CUDA(cudaMemcpyToSymbolAsync(umma::g_wait_ns, &ns, sizeof(ns), 0, cudaMemcpyHostToDevice, st));
  NED_CUDA(cudaStreamSynchronize(st));
  return oz64_set_wait_ns(ns, st);
}

}  // namespace nedmft

// ------------------------------------------------------------------ small GEMMs of the warm-start network
//
// C[m x n] = op(A) op(B) (+ bias[n]) (+ C), FP32 in memory: op(A) is m x k
// (ta: A stored k x m, else m x k, both row-major), op(B) is k x n (tb: B
// stored n x k, else k x n).  Each CTA takes 128 rows of C and all n <= 256
// columns; the operands of a 64-deep K chunk are rounded to bf16 into shared
// memory in the canonical K-major layout by all 128 threads (zeros past m, n
// and k), one thread issues the tcgen05 products (M = 128, N = n rounded up
// to 16) into an FP32 TMEM accumulator, two chunk buffers alternate.  With
// gridDim.y > 1 each CTA sums a contiguous part of K into its own slice of
// `part` (m x n each) and mlp_split_reduce_kernel adds the slices in order.
namespace nedmft {
namespace {

constexpr int kMlpK = 64;  // K per chunk

__global__ void __launch_bounds__(128, 1)
    mlp_umma_gemm_kernel(const float* __restrict__ A, const float* __restrict__ B, const float* __restrict__ bias,
                         float* __restrict__ C, float* __restrict__ part, int m, int n, int k, bool ta, bool tb,
                         bool accumulate, int chunks_per_split, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int np16 = (n + 15) & ~15;
  const int nrows_b = (np16 + 127) & ~127;  // B rows held (1 or 2 tiles of 128)
  const int a_bytes = kTileBytes, b_bytes = nrows_b / 128 * kTileBytes;
  const int stage = a_bytes + b_bytes;
  uint64_t* done = reinterpret_cast<uint64_t*>(smem + 2 * stage);  // [2] chunk products complete, [2] all complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int row0 = blockIdx.x * 128;
  const int nchunks = (k + kMlpK - 1) / kMlpK;
  const int c_begin = blockIdx.y * chunks_per_split;
  const int c_end = min(nchunks, c_begin + chunks_per_split);
  uint32_t cols = 32;
  while ((int)cols < np16) cols <<= 1;
  if (t == 0) {
    mbar_init(&done[0], 1);
    mbar_init(&done[1], 1);
    mbar_init(&done[2], 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_bf16(128, np16);
  bool ok = true;
  int issued = 0;
  for (int c = c_begin; c < c_end; ++c) {
    const int s = (c - c_begin) & 1;
    unsigned char* st = smem + s * stage;
    if (c - c_begin >= 2) {  // the products that read this buffer two chunks ago are done
      if (!__syncthreads_and(mbar_wait(&done[s], (((c - c_begin) >> 1) - 1) & 1, abort_flag))) { ok = false; break; }
    }
    __nv_bfloat16* sa = reinterpret_cast<__nv_bfloat16*>(st);
    __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(st + a_bytes);
    const int k0 = c * kMlpK;
    for (int e = t; e < 128 * kMlpK; e += 128) {
      const int r = ta ? (e & 127) : (e >> 6), kk = ta ? (e >> 7) : (e & 63);
      const int gr = row0 + r, gk = k0 + kk;
      float v = 0.f;
      if (gr < m && gk < k) v = ta ? A[(size_t)gk * m + gr] : A[(size_t)gr * k + gk];
      sa[img_offset(r, kk, 1)] = __float2bfloat16_rn(v);
    }
    for (int e = t; e < nrows_b * kMlpK; e += 128) {
      const int j = tb ? (e >> 6) : (e % nrows_b), kk = tb ? (e & 63) : (e / nrows_b);
      const int gk = k0 + kk;
      float v = 0.f;
      if (j < n && gk < k) v = tb ? B[(size_t)j * k + gk] : B[(size_t)gk * n + j];
      sb[img_offset(j, kk, 1)] = __float2bfloat16_rn(v);
    }
    fence_proxy_async();  // the generic stores above become visible to the tensor core
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      const uint32_t a_addr = smem_u32(sa), b_addr = smem_u32(sb);
#pragma unroll
      for (int kk = 0; kk < kMlpK / 16; ++kk)
        mma_bf16(tmem, smem_desc(a_addr + kk * 256, 128, 1024), smem_desc(b_addr + kk * 256, 128, 1024), idesc,
                 (c > c_begin || kk > 0) ? 1u : 0u);
      mma_commit(&done[s]);
    }
    ++issued;
  }
  if (t == 0) mma_commit(&done[2]);  // after every product issued above (also after an abort)
  // every thread: the accumulator is complete (bounded by the drain limit)
  {
    const uint64_t t0 = global_ns();
    while (!mbar_test(&done[2], 0) && global_ns() - t0 < kDrainNs) {
    }
  }
  tc_fence_after();
  if (ok && issued > 0) {
    const int r = row0 + warp * 32 + lane;
    for (int c0 = 0; c0 < np16; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
      if (r < m) {
        if (gridDim.y > 1) {
          float* out = part + ((size_t)blockIdx.y * m + r) * n;
#pragma unroll
          for (int e = 0; e < 32; ++e)
            if (c0 + e < n) out[c0 + e] = v[e];
        } else {
          float* out = C + (size_t)r * n;
#pragma unroll
          for (int e = 0; e < 32; ++e)
            if (c0 + e < n) {
              float x = v[e] + (bias ? bias[c0 + e] : 0.f);
              if (accumulate) x += out[c0 + e];
              out[c0 + e] = x;
            }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, cols);
  }
  if (t == 0 && *abort_flag && status) atomicCAS(status, 0, DS_TIMEOUT);
}

// C = sum over the slices of part (in order) (+ bias) (+ C)
__global__ void mlp_split_reduce_kernel(const float* __restrict__ part, int splits, const float* __restrict__ bias,
                                        float* __restrict__ C, int m, int n, bool accumulate) {
  const size_t total = (size_t)m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    float x = 0.f;
    for (int s = 0; s < splits; ++s) x += part[(size_t)s * total + e];
    if (bias) x += bias[e % n];
    if (accumulate) x += C[e];
    C[e] = x;
  }
}

}  // namespace

size_t umma_mlp_split_bytes(int m, int n, int splits) { return sizeof(float) * (size_t)m * n * splits; }

int umma_mlp_gemm(const float* A, const float* B, const float* bias, float* C, int m, int n, int k, bool ta, bool tb,
                  bool accumulate, float* part, int splits, cudaStream_t st) {
  if (n < 1 || n > 256 || m < 1 || k < 1) return set_error(NEDMFT_EINVAL, "mlp gemm: shape %d x %d x %d", m, n, k);
  const int nchunks = (k + kMlpK - 1) / kMlpK;
  if (splits < 1 || !part) splits = 1;
  if (splits > nchunks) splits = nchunks;
  const int cps = (nchunks + splits - 1) / splits;
  splits = (nchunks + cps - 1) / cps;
  const int np16 = (n + 15) & ~15, nrows_b = (np16 + 127) & ~127;
  const int smem = 2 * (kTileBytes + nrows_b / 128 * kTileBytes) + 1024 + 64;
  int rc = ensure_dyn_smem(reinterpret_cast<const void*>(mlp_umma_gemm_kernel), smem);
  if (rc) return rc;
  int* status = device_status_ptr();
  mlp_umma_gemm_kernel<<<dim3((m + 127) / 128, splits), 128, smem, st>>>(A, B, bias, C, part, m, n, k, ta, tb,
                                                                        accumulate, cps, status);
  NED_LAUNCH_CHECK("mlp_umma_gemm_kernel");
  if (splits > 1) {
    const size_t total = (size_t)m * n;
    const int blocks = (int)((total + 255) / 256 < 1216 ? (total + 255) / 256 : 1216);
    mlp_split_reduce_kernel<<<blocks, 256, 0, st>>>(part, splits, bias, C, m, n, accumulate);
    NED_LAUNCH_CHECK("mlp_split_reduce_kernel");
  }
  return NEDMFT_OK;
}

}  // namespace nedmft
