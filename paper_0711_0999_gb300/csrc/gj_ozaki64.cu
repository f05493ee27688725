// FP64-accurate trailing update of the pivoted Gauss-Jordan inversion (the
// impurity step) on the tensor cores:  A <- A (rows and columns of the block K
// zeroed) - C R  with C = A_{:,K} (np x 32 complex) and R = P A_{K,:} (32 x np).
//
// Ozaki split: every row of C (64 reals, re and im interleaved over k) and
// every row of the 2 x 2 real embedding of R (output column n, 64 reals) is
// scaled by a power of two to below one and cut into kOz64S integer slices
// of 7 bits (balanced base-128 digits of x 2^-e), so x = 2^e sum_s q_s
// 2^-7(s+1) up to 2^-7 kOz64S.  A slice product sum_k q_a q_b is below 2^21 and
// the up-to-7 products of one order o = a + b below 2^23, so bf16 operands
// with FP32 accumulation in TMEM give every order's sum exactly.  The 28
// products of order <= 6 leave a truncation near 1e-15 of the row and column
// maxima (FP64 level); the epilogue adds the order sums, scaled by
// 2^-7(o+2), in double-float (FP32 pairs, 48 bits) and subtracts the result
// from A in FP64.
#include "lattice.cuh"
#include "umma_core.cuh"

namespace nedmft {

using namespace umma;

namespace {

constexpr int kOz64S = 7;     // slices per operand
constexpr int kOz64Bits = 7;  // bits per slice
constexpr int kOz64K = 64;    // K of the rank-32 complex update (re, im interleaved)
constexpr int kOz64Bn = 64;   // output real columns per tile
constexpr int kOz64Orders = kOz64S;  // orders 0 .. kOz64S - 1 are kept

__device__ __forceinline__ void two_sum64(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// The slices of one row (64 reals, lane l holding k = 2l, 2l+1): the row
// exponent e (max |x| < 2^e) from a warp maximum, then X = round(x 2^(49-e)),
// |X| < 2^49, cut into balanced base-128 digits from the bottom (six digits
// in [-64, 63], the top one the rest, |q_0| <= 129; all exact in bf16), so
// x = 2^e sum_s q_s 2^-7(s+1) up to 2^(e-50).  Integer work except two FP64
// operations per value.
__device__ __forceinline__ void oz64_slice_row(double v0, double v1, int row, int lane, __nv_bfloat16* img,
                                               size_t slice, int* ex) {
  double m = fmax(fabs(v0), fabs(v1));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  int e = 0;
  if (m > 0.0) frexp(m, &e);  // m < 2^e
  if (lane == 0) ex[row] = e;
  constexpr int kTop = kOz64Bits * kOz64S;  // 49
  long long x0 = llrint(ldexp(v0, kTop - e)), x1 = llrint(ldexp(v1, kTop - e));
  int q0[kOz64S], q1[kOz64S];
#pragma unroll
  for (int s = kOz64S - 1; s > 0; --s) {
    const int d0 = (int)((x0 + 64) & 127) - 64, d1 = (int)((x1 + 64) & 127) - 64;
    q0[s] = d0;
    q1[s] = d1;
    x0 = (x0 - d0) >> kOz64Bits;
    x1 = (x1 - d1) >> kOz64Bits;
  }
  q0[0] = (int)x0;
  q1[0] = (int)x1;
  const size_t o = img_offset(row, 2 * lane, 1);
#pragma unroll
  for (int s = 0; s < kOz64S; ++s)
    *reinterpret_cast<__nv_bfloat162*>(img + s * slice + o) =
        __halves2bfloat162(__float2bfloat16_rn((float)q0[s]), __float2bfloat16_rn((float)q1[s]));
}

// Slices of the rows of C (np rows, blocks 0 .. np/8 - 1: a warp per row) and
// of the embedded R (2 np rows, blocks np/8 .. : 32 columns j of R per block,
// read by rows of R into shared memory, then a warp per pair of rows 2j, 2j+1).
// Row images in the canonical K-major layout (one 128-row tile of 64 k per
// 128 rows), slice s at s * slice.
__global__ void __launch_bounds__(256) oz64_pack_kernel(const double2* __restrict__ Rbuf,
                                                        const double2* __restrict__ Cbuf, int np,
                                                        __nv_bfloat16* __restrict__ cimg, int* __restrict__ cexp,
                                                        __nv_bfloat16* __restrict__ rimg, int* __restrict__ rexp) {
  __shared__ double2 tile[32][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cblocks = np / 8;
  if ((int)blockIdx.x < cblocks) {  // row i of C: (Re, Im) of C[i][lane]
    const int i = blockIdx.x * 8 + warp;
    const double2 z = Cbuf[(size_t)i * 32 + lane];
    oz64_slice_row(z.x, z.y, i, lane, cimg, (size_t)np * kOz64K, cexp);
    return;
  }
  const int j0 = (blockIdx.x - cblocks) * 32;
  for (int c = warp; c < 32; c += 8) tile[c][lane] = Rbuf[(size_t)c * np + j0 + lane];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int jj = 4 * warp + q, j = j0 + jj;
    const double2 z = tile[lane][jj];  // R[c = lane][j]
    oz64_slice_row(z.x, -z.y, 2 * j, lane, rimg, (size_t)2 * np * kOz64K, rexp);     // [re, -im]
    oz64_slice_row(z.y, z.x, 2 * j + 1, lane, rimg, (size_t)2 * np * kOz64K, rexp);  // [im, re]
  }
}

struct Oz64Smem {
  static constexpr int kA = kOz64S * kTileBytes;      // 128 rows x 64 k per slice
  static constexpr int kB = kOz64S * kTileBytes / 2;  // 64 rows x 64 k per slice
  static constexpr int kBytes = kA + kB + 1024 /*align*/ + 64 /*barriers*/;
};

// SMs left to the kernels of the look-ahead stream while the update runs (the
// tournament's CTAs need more shared memory than an update CTA leaves free).
constexpr int kOz64FreeSms = 8;

// x as a double, exactly, on the integer units (IEEE 754 binary32 to binary64:
// the exponent rebiased by 1023 - 127 = 896, the 23 fraction bits moved up by
// 29); zero keeps its sign.  Subnormal, infinite and NaN values, which an order
// sum scaled inside the FP32 range does not produce, take the conversion
// instruction.  GB300 runs conversions on its two FP64 units per SM.
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = __float_as_uint(x), a = u & 0x7fffffffu;
  if (a - 0x00800000u >= 0x7f000000u) {  // zero, subnormal, infinity or NaN
    if (a == 0) return __hiloint2double((int)u, 0);
    return (double)x;
  }
  return __hiloint2double((int)((u & 0x80000000u) | ((a >> 3) + (896u << 20))), (int)(u << 29));
}

// Persistent over the output tiles (128 rows, 64 real columns = 32 complex) of
// the np x 2np real image of A, row-tile major, a contiguous run of tiles per
// CTA, so consecutive tiles mostly share their 128 rows: the A slices are
// brought in once per row tile.  Per tile thread 0 brings the 7 B (and, for a
// new row tile, 7 A) slice blocks in with bulk copies, then issues the 28
// products of order <= 6 (4 MMAs of K = 16 each) into 7 order accumulators of
// 64 TMEM columns; 8 warps drain them (one TMEM lane per row, two warps per
// lane quarter, 32 columns each).  Column j of A is written iff
// (wlo <= j < whi) == inside (the look-ahead window: see pivot_inverse).
__global__ void __launch_bounds__(256, 1) oz64_update_kernel(double2* __restrict__ A, int np, int k0,
                                                             const __nv_bfloat16* __restrict__ cimg,
                                                             const int* __restrict__ cexp,
                                                             const __nv_bfloat16* __restrict__ rimg,
                                                             const int* __restrict__ rexp, int wlo, int whi,
                                                             bool inside, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* sa = smem;
  unsigned char* sb = smem + Oz64Smem::kA;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Oz64Smem::kA + Oz64Smem::kB);  // [0] loads, [1] products
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int ntn = 2 * np / kOz64Bn, ntiles = (np / 128) * ntn;
  const int tile_lo = (int)((long long)blockIdx.x * ntiles / gridDim.x);
  const int tile_hi = (int)((long long)(blockIdx.x + 1) * ntiles / gridDim.x);
  constexpr uint32_t kCols = 512;  // 7 x 64 columns, allocated as a power of two
  if (t == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, kCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const size_t cslice = (size_t)np * kOz64K, rslice = (size_t)2 * np * kOz64K;
  // the next tile at or after `tile` that writes any column (or tile_hi)
  auto next_active = [&](int tile) {
    for (; tile < tile_hi; ++tile) {
      const int j_lo = (tile % ntn) * (kOz64Bn / 2), j_hi = j_lo + kOz64Bn / 2;
      const bool skip = inside ? (j_hi <= wlo || j_lo >= whi) : (j_lo >= wlo && j_hi <= whi);
      if (!skip) break;
    }
    return tile;
  };
  int cur_mt = -1;  // the row tile whose A slices are (being) brought into shared memory
  // thread 0: the operands of `tile` (the B slices, and the A slices of a new row tile) on bars[0]
  auto load = [&](int tile) {
    const int mt = tile / ntn, n0 = (tile % ntn) * kOz64Bn;
    const bool load_a = mt != cur_mt;
    cur_mt = mt;
    if (t != 0) return;
    mbar_arrive_expect_tx(&bars[0], (load_a ? Oz64Smem::kA : 0) + Oz64Smem::kB);
    for (int s = 0; s < kOz64S; ++s) {
      // the canonical image: 128-row tile mt of slice s (16 KB); 64 rows of
      // tile n0 / 128 starting at row n0 % 128 (8 KB, 8-row groups contiguous)
      if (load_a) bulk_g2s(sa + s * kTileBytes, cimg + s * cslice + (size_t)mt * kTileElems, kTileBytes, &bars[0]);
      bulk_g2s(sb + s * (kTileBytes / 2), rimg + s * rslice + (size_t)(n0 >> 7) * kTileElems + (size_t)(n0 & 127) * 64,
               kTileBytes / 2, &bars[0]);
    }
  };
  uint32_t it = 0;  // tiles done: the phase parity of both barriers
  bool ok = true;
  int tile = next_active(tile_lo);
  if (tile < tile_hi) load(tile);
  while (tile < tile_hi && ok) {
    const int mt = tile / ntn, n0 = (tile % ntn) * kOz64Bn;  // 128-row tile, first real column (2 j0)
    const uint32_t par = it & 1u;
    ok = __syncthreads_and(mbar_wait(&bars[0], par, abort_flag));
    if (ok && t == 0) {
      tc_fence_after();
      constexpr uint32_t idesc = idesc_bf16(128, kOz64Bn);
      for (int a = 0; a < kOz64S; ++a)
        for (int b = 0; a + b < kOz64Orders; ++b)
#pragma unroll
          for (int kk = 0; kk < kOz64K / 16; ++kk)
            mma_bf16(tmem + (uint32_t)(a + b) * kOz64Bn,
                     smem_desc(smem_u32(sa + a * kTileBytes) + kk * 256, 128, 1024),
                     smem_desc(smem_u32(sb + b * (kTileBytes / 2)) + kk * 256, 128, 1024), idesc,
                     (a > 0 || kk > 0) ? 1u : 0u);
    }
    if (t == 0) mma_commit(&bars[1]);  // after every product issued above (also after a failed load wait)
    bool done;
    {
      const uint64_t t0 = global_ns();
      while (!(done = mbar_test(&bars[1], par)) && global_ns() - t0 < kDrainNs) {
      }
      // no copy may be left in flight at exit (only after a failed wait)
      if (!ok && t == 0)
        while (!mbar_test(&bars[0], par) && global_ns() - t0 < kDrainNs) {
        }
    }
    if (!done) *abort_flag = 1;
    ok = __syncthreads_and(ok && done);
    tc_fence_after();
    const int next = ok ? next_active(tile + 1) : tile_hi;
    // the products have read the operands: the next tile's come in during this epilogue
    if (next < tile_hi) load(next);
    if (ok) {
      const int i = mt * 128 + (warp & 3) * 32 + lane;  // this thread's row (TMEM lane)
      const bool ik = i >= k0 && i < k0 + 32;
      const int ei = cexp[i];
      const int c0 = 32 * (warp >> 2);  // warps 0-3 and 4-7 drain the two 32-column halves
      float hi[32], lo[32];
      tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + c0, hi);
#pragma unroll
      for (int u = 0; u < 32; ++u) lo[u] = 0.f;
      for (int o = 1; o < kOz64Orders; ++o) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)o * kOz64Bn + c0, v);
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          float s, e;
          two_sum64(hi[u], ldexpf(v[u], -kOz64Bits * o), s, e);
          hi[u] = s;
          lo[u] += e;
        }
      }
      // the accumulators are read (ordered before the barrier after which the
      // next tile's products overwrite them)
      tc_fence_before();
#pragma unroll
      for (int u = 0; u < 32; u += 2) {
        const int n = n0 + c0 + u, j = n >> 1;
        if ((j >= wlo && j < whi) != inside) continue;
        const bool jk = j >= k0 && j < k0 + 32;
        // order sums carry 2^-7(o+2) 2^(ei + en): o is in the ldexpf above.
        // The power of two is applied in FP32 (exact) while the result stays
        // well inside the FP32 range, then two exact conversions on the
        // integer units and two FP64 subtractions per value; else in FP64
        const int s0 = ei + rexp[n] - 2 * kOz64Bits, s1 = ei + rexp[n + 1] - 2 * kOz64Bits;
        double2* a = A + (size_t)i * np + j;
        double2 nv = (ik || jk) ? make_double2(0.0, 0.0) : *a;
        if (s0 > -64 && s0 < 64) {
          nv.x = (nv.x - f32_to_f64(ldexpf(hi[u], s0))) - f32_to_f64(ldexpf(lo[u], s0));
        } else {
          nv.x -= ldexp((double)hi[u] + (double)lo[u], s0);
        }
        if (s1 > -64 && s1 < 64) {
          nv.y = (nv.y - f32_to_f64(ldexpf(hi[u + 1], s1))) - f32_to_f64(ldexpf(lo[u + 1], s1));
        } else {
          nv.y -= ldexp((double)hi[u + 1] + (double)lo[u + 1], s1);
        }
        *a = nv;
      }
    }
    ++it;
    tile = next;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kCols);
  }
  if (t == 0 && *abort_flag && status) atomicCAS(status, 0, DS_TIMEOUT);
}

}  // namespace

size_t oz64_workspace(int np) {
  return align256(sizeof(__nv_bfloat16) * (size_t)kOz64S * np * kOz64K) +
         align256(sizeof(__nv_bfloat16) * (size_t)kOz64S * 2 * np * kOz64K) + align256(sizeof(int) * (size_t)np) +
         align256(sizeof(int) * (size_t)2 * np);
}

// Limit of the bounded waits of this file's kernel on the current device
// (stream-ordered after earlier work on `st`).
int oz64_set_wait_ns(uint64_t ns, cudaStream_t st) {
  NED_CUDA(cudaMemcpyToSymbolAsync(umma::g_wait_ns, &ns, sizeof(ns), 0, cudaMemcpyHostToDevice, st));
  NED_CUDA(cudaStreamSynchronize(st));
  return NEDMFT_OK;
}

// The kernel's shared-memory limit and the device's SM count (which sizes its
// grid), both cached per device: called before a graph capture of oz64_update.
int oz64_prepare() {
  int sms = 0;
  if (int rc = device_sm_count(&sms)) return rc;
  return ensure_dyn_smem(reinterpret_cast<const void*>(oz64_update_kernel), Oz64Smem::kBytes);
}

int oz64_update(double2* A, int np, int k0, const double2* Rbuf, const double2* Cbuf, int wlo, int whi, bool inside,
                void* ws, cudaStream_t st, int* status) {
  if (np % 128) return set_error(NEDMFT_EINVAL, "oz64_update: np = %d not a multiple of 128", np);
  char* p = static_cast<char*>(ws);
  __nv_bfloat16* cimg = reinterpret_cast<__nv_bfloat16*>(p);
  p += align256(sizeof(__nv_bfloat16) * (size_t)kOz64S * np * kOz64K);
  __nv_bfloat16* rimg = reinterpret_cast<__nv_bfloat16*>(p);
  p += align256(sizeof(__nv_bfloat16) * (size_t)kOz64S * 2 * np * kOz64K);
  int* cexp = reinterpret_cast<int*>(p);
  p += align256(sizeof(int) * (size_t)np);
  int* rexp = reinterpret_cast<int*>(p);
  oz64_pack_kernel<<<np / 8 + np / 32, 256, 0, st>>>(Rbuf, Cbuf, np, cimg, cexp, rimg, rexp);
  NED_LAUNCH_CHECK("oz64_pack_kernel");
  if (int rc = oz64_prepare()) return rc;
  int sms = 0;
  if (int rc = device_sm_count(&sms)) return rc;
  const int tiles = (np / 128) * (2 * np / kOz64Bn);
  int grid = sms > 2 * kOz64FreeSms ? sms - kOz64FreeSms : sms;
  if (grid > tiles) grid = tiles;
  oz64_update_kernel<<<grid, 256, Oz64Smem::kBytes, st>>>(A, np, k0, cimg, cexp, rimg, rexp, wlo, whi, inside,
                                                          status);
  NED_LAUNCH_CHECK("oz64_update_kernel");
  return NEDMFT_OK;
}

}  // namespace nedmft
