// Persistent TMA-fed tensor-core kernel for the mode products of the BP sweep
// and the gate (Eq. MessageTensorSelfConsistency contracted leg by leg):
//   Y[m][(t, n)] = sum_(s, k) A_s[m][k] Bt[(t, n)][(s, k)],
// A a site-shaped planar complex tensor whose rows m (all legs but the
// contracted one, and p) are streamed once, Bt the realified transposed
// chi x chi message (a real [2 chi][2 chi] matrix, the same for every row of
// one site).  With chi = 64 one site is 64 tiles of 128 rows; the operand
// streams at HBM rate while the tensor core does 4.2 MFLOP per 128 KB of
// traffic, so the kernel is bound by HBM, not by the tensor pipe.
//
// One CTA per SM walks a contiguous range of (site, row tile) pairs:
//   warp 0 (one thread)  TMA producer: the site's Bt once per site (4 chunks
//                        of [2 chi rows][32 floats], 128-byte swizzle), then
//                        per tile the 2 chi / 32 K chunks of A, [128 rows][32
//                        floats] each, into an 8-slot ring (full / empty
//                        mbarriers, transaction counts);
//   warp 1 (one thread)  tcgen05.mma (M = 128, N = 2 chi, K = 8 TF32) into one
//                        of two TMEM accumulators, commits release the ring
//                        slot, the accumulator and, at a site change, Bt;
//   warps 2..5           epilogue: tcgen05.ld of their 32-lane quadrant,
//                        coalesced stores (consecutive rows are consecutive
//                        addresses in every output layout the engine builds),
//                        then release the accumulator, so the store of tile i
//                        overlaps the loads and MMAs of tile i + 1.
// The A rows are addressed by a TMA tensor map over (k, up to three row
// levels, plane); the engine encodes one map per site when it builds a plan.
// Every mbarrier wait is bounded (about one second): on expiry the kernel sets
// bit 1 of *err, stops issuing, waits (bounded) for the copies and MMAs it has
// in flight and frees its tensor memory.
#include <cuda.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "tc_common.cuh"
#include "tnbp.h"

namespace tnbp {
namespace {

using namespace tc;

constexpr int kThreads = 192;
constexpr int kSlots = 8;                 // A ring: 8 x 16 KB
constexpr int kChunk = 128 * 128;         // one [128 rows][128 bytes] chunk
constexpr int kBBytes = 4 * kChunk;       // Bt: up to 4 chunks of [128 rows][128 bytes]
constexpr int kBarOff = kBBytes + kSlots * kChunk;
constexpr int kSmemBytes = kBarOff + 256 + 1024;  // barriers + alignment slack

struct StreamArgs {
  const CUtensorMap* maps;  // [2 * n_outer]: A maps, then Bt maps
  int n_outer;
  int tiles_per_entry;      // M / 128
  int kc;                   // K chunks of 32 floats: 2 chi / 32
  int nr;                   // real N: 2 chi
  int chi;
  int rank;                 // A map rank: 2 + number of row levels
  int lev0, lev1;           // sizes of the two innermost row levels (for coordinates)
  int* err;
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, int c4, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
      "r"(smem_u32(bar))
      : "memory");
}

__global__ void __launch_bounds__(kThreads, 1) tc_stream_kernel(GemmDesc d, StreamArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sB = smem;
  unsigned char* sA = smem + kBBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kBarOff);
  uint64_t* empty = full + kSlots;
  uint64_t* bfull = empty + kSlots;
  uint64_t* bempty = bfull + 1;
  uint64_t* tfull = bempty + 1;   // [2]
  uint64_t* tempty = tfull + 2;   // [2]
  uint64_t* done = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int total = a.n_outer * a.tiles_per_entry;
  const int t_beg = (int)((int64_t)blockIdx.x * total / gridDim.x);
  const int t_end = (int)((int64_t)(blockIdx.x + 1) * total / gridDim.x);
  const uint32_t tmem_cols = 2 * a.nr;  // two accumulators of nr columns (128 or 256)

  if (tid == 0) {
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(bfull, 1);
    mbar_init(bempty, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const CUtensorMap* amaps = a.maps;
  const CUtensorMap* bmaps = a.maps + a.n_outer;

  if (warp == 0) {
    // ------------------------------------------------------------- producer
    if (lane == 0) {
      int it = 0, cur = -1, bl = 0;
      int issued[kSlots];
#pragma unroll
      for (int s = 0; s < kSlots; ++s) issued[s] = 0;
      const uint32_t bbytes = (uint32_t)(a.kc * a.nr * 128);
      for (int tile = t_beg; tile < t_end && !*abort_flag; ++tile) {
        const int e = tile / a.tiles_per_entry;
        if (outer_frozen(d, e)) continue;  // every role skips the same tiles
        const int mt = tile - e * a.tiles_per_entry;
        if (e != cur) {
          if (cur >= 0 && !mbar_wait(bempty, (bl - 1) & 1, a.err)) { *abort_flag = 1; break; }
          mbar_expect_tx(bfull, bbytes);
          for (int c = 0; c < a.kc; ++c)
            tma_load_2d(smem_u32(sB + c * a.nr * 128), bmaps + e, c * 32, 0, bfull);
          ++bl;
          cur = e;
        }
        // row coordinates of the tile's first row in the map's row levels
        int r = mt * 128;
        const int r0 = r % a.lev0;
        r /= a.lev0;
        const int r1 = r % a.lev1;
        const int r2 = r / a.lev1;
        for (int c = 0; c < a.kc; ++c, ++it) {
          const int slot = it % kSlots;
          if (!mbar_wait(&empty[slot], ((it / kSlots) & 1) ^ 1, a.err)) { *abort_flag = 1; break; }
          mbar_expect_tx(&full[slot], (uint32_t)kChunk);
          const int kr = c * 32, plane = kr / a.chi, k = kr - plane * a.chi;
          const uint32_t dst = smem_u32(sA + slot * kChunk);
          if (a.rank == 3) tma_load_3d(dst, amaps + e, k, r0, plane, &full[slot]);
          else if (a.rank == 4) tma_load_4d(dst, amaps + e, k, r0, r1, plane, &full[slot]);
          else tma_load_5d(dst, amaps + e, k, r0, r1, r2, plane, &full[slot]);
          ++issued[slot];
        }
      }
      // before the CTA exits: every copy issued has landed (immediate on the
      // normal path, where the consumer already waited for each of them)
      for (int s = 0; s < kSlots; ++s)
        if (issued[s] > 0) mbar_wait(&full[s], (issued[s] - 1) & 1, a.err);
      if (bl > 0) mbar_wait(bfull, (bl - 1) & 1, a.err);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t idesc = make_idesc(2, 128, a.nr);
      int it = 0, cur = -1, bl = 0, i = 0;  // i: tiles processed (the skipped ones not counted)
      for (int tile = t_beg; tile < t_end && !*abort_flag; ++tile) {
        const int e = tile / a.tiles_per_entry;
        if (outer_frozen(d, e)) continue;
        if (e != cur) {
          if (cur >= 0) mma_commit(bempty);  // arrives once the MMAs reading Bt are done
          if (!mbar_wait(bfull, bl & 1, a.err)) { *abort_flag = 1; break; }
          ++bl;
          cur = e;
        }
        const int acc = i & 1;
        if (!mbar_wait(&tempty[acc], ((i >> 1) & 1) ^ 1, a.err)) { *abort_flag = 1; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem + (uint32_t)(acc * a.nr);
        bool ok = true;
        for (int c = 0; c < a.kc; ++c, ++it) {
          const int slot = it % kSlots;
          if (!mbar_wait(&full[slot], (it / kSlots) & 1, a.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + slot * kChunk);
          const uint32_t b0 = smem_u32(sB + c * a.nr * 128);
          // descriptors of the chunk; a 32-byte K step adds 2 to the start field
          const uint64_t da = sw128_desc(a0), db = sw128_desc(b0);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            mma_issue(0, d_tmem, da + 2 * ks, db + 2 * ks, idesc,
                      (c > 0 || ks > 0) ? 1u : 0u);
          mma_commit(&empty[slot]);
        }
        if (!ok) { *abort_flag = 1; break; }
        mma_commit(&tfull[acc]);
        ++i;
      }
      // all MMAs issued by this thread complete before TMEM is freed
      mma_commit(done);
      mbar_wait(done, 0, a.err);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const int row = q * 32 + lane;
    int i = 0;  // tiles processed (the skipped ones not counted)
    for (int tile = t_beg; tile < t_end; ++tile) {
      if (*abort_flag) break;
      const int e = tile / a.tiles_per_entry;
      if (outer_frozen(d, e)) continue;
      const int mt = tile - e * a.tiles_per_entry;
      const int acc = i & 1;
      const bool ok = mbar_wait(&tfull[acc], (i >> 1) & 1, a.err);
      if (!ok) { *abort_flag = 1; break; }
      tc_fence_after();
      __syncwarp();
      const int m = mt * 128 + row;
      float* C = d.C[e] + ROW_C(d, m);
      for (int c0 = 0; c0 < a.nr; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * a.nr + c0), v);
        const int t = c0 >= a.chi;
        float* Cc = C + (t ? d.plane_c : 0) + (int64_t)(c0 - t * a.chi) * d.c_n;
        if (d.c_n == 1) {
          // columns contiguous in the output: 16-byte stores along the row
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            *reinterpret_cast<float4*>(Cc + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        } else {
          // rows contiguous: lane-consecutive addresses, one 128-byte store per column
#pragma unroll
          for (int j = 0; j < 32; ++j) Cc[(int64_t)j * d.c_n] = v[j];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
      ++i;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------- closes
// out[m][n] = sum_K A[m][K] op(B[n][K]) with M = N = 64 (the message's two
// indices), both operands K-contiguous site tensors: per K chunk of 32 the
// tile is [(s, m)][32] of A and [(t, n)][32] of B (s, t the re/im planes, so
// the 128 x 128 product holds all four real products P_st), streamed by TMA
// through a 3-stage ring; K is split over CTAs, two CTAs per SM.  The
// epilogue stages P in shared memory, combines C_re = P_rr - sa sb P_ii,
// C_im = sb P_ri + sa P_ir and writes the CTA's partial; a second kernel sums
// the partials in a fixed order.  With one split the CTA writes the output
// itself and no reduce runs.
constexpr int kCThreads = 192;
constexpr int kCStages = 3;
constexpr int kCStage = 2 * kChunk;  // A 16 KB + B 16 KB
constexpr int kCBarOff = kCStages * kCStage;
constexpr int kCSmemBytes = kCBarOff + 128 + 1024;

struct CloseArgs {
  const CUtensorMap* maps;  // [2 * n_outer]: A maps, then B maps
  int n_outer, chunks, per_split, K2;
  int direct;               // one split: the output is written here, no partials
  float* part;
  int* err;
};

__global__ void __launch_bounds__(kCThreads, 2) tc_close_kernel(GemmDesc d, CloseArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kCBarOff);
  uint64_t* empty = full + kCStages;
  uint64_t* accum = empty + kCStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int e = blockIdx.y, split = blockIdx.x;
  // a converged component of a union: nothing is initialised yet, the whole
  // CTA leaves together (its partial is never read: the reduce skips it too)
  if (outer_frozen(d, e / d.n_inner)) return;
  const int c0 = split * a.per_split;
  const int c1 = min(a.chunks, c0 + a.per_split);
  const int nt = c1 > c0 ? c1 - c0 : 0;  // >= 1 by the host's choice of splits

  if (tid == 0) {
    for (int s = 0; s < kCStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const CUtensorMap* amap = a.maps + e;
  const CUtensorMap* bmap = a.maps + a.n_outer + e;

  if (warp == 0) {
    if (lane == 0) {
      int issued[kCStages] = {0, 0, 0};
      for (int i = 0; i < nt && !*abort_flag; ++i) {
        const int slot = i % kCStages;
        if (!mbar_wait(&empty[slot], ((i / kCStages) & 1) ^ 1, a.err)) { *abort_flag = 1; break; }
        mbar_expect_tx(&full[slot], (uint32_t)(2 * kChunk));
        const int k = (c0 + i) * 32;
        const int k1 = k / a.K2, k2 = k - k1 * a.K2;
        const uint32_t dst = smem_u32(smem + slot * kCStage);
        tma_load_4d(dst, amap, k2, 0, k1, 0, &full[slot]);
        tma_load_4d(dst + kChunk, bmap, k2, 0, k1, 0, &full[slot]);
        ++issued[slot];
      }
      for (int s = 0; s < kCStages; ++s)
        if (issued[s] > 0) mbar_wait(&full[s], (issued[s] - 1) & 1, a.err);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = make_idesc(2, 128, 128);
      for (int i = 0; i < nt && !*abort_flag; ++i) {
        const int slot = i % kCStages;
        if (!mbar_wait(&full[slot], (i / kCStages) & 1, a.err)) { *abort_flag = 1; break; }
        tc_fence_after();
        const uint32_t a0 = smem_u32(smem + slot * kCStage);
        // descriptors of the chunk; a 32-byte K step adds 2 to the start field
        const uint64_t da = sw128_desc(a0), db = sw128_desc(a0 + kChunk);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          mma_issue(0, tmem, da + 2 * ks, db + 2 * ks, idesc,
                    (i > 0 || ks > 0) ? 1u : 0u);
        mma_commit(&empty[slot]);
      }
      mma_commit(accum);  // also orders TMEM release after every MMA issued
    }
    __syncwarp();
  }
  // every thread: the accumulator is final (or the CTA gave up)
  const bool ok = mbar_wait(accum, 0, a.err) && !*abort_flag && nt > 0;
  tc_fence_after();
  if (warp >= 2) {
    // P staged in the (now idle) pipeline buffers: [128 rows][129]
    float* P = reinterpret_cast<float*>(smem);
    const int q = warp & 3, row = q * 32 + lane;
#pragma unroll
    for (int c = 0; c < 128; c += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) P[row * 129 + c + j] = v[j];
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    const float sa = d.conj_a ? -1.f : 1.f, sb = d.conj_b ? -1.f : 1.f;
    float* out = a.part + ((int64_t)split * a.n_outer + e) * 2 * 4096;
    const int outer = e / d.n_inner, inner = e - outer * d.n_inner;
    float* C = d.C[outer] + inner * d.c_in;
    for (int idx = tid - 64; idx < 4096; idx += 128) {
      const int m = idx >> 6, n = idx & 63;
      float cr = 0.f, ci = 0.f;
      if (ok) {
        const float prr = P[m * 129 + n], pii = P[(64 + m) * 129 + 64 + n];
        const float pri = P[m * 129 + 64 + n], pir = P[(64 + m) * 129 + n];
        cr = prr - sa * sb * pii;
        ci = sb * pri + sa * pir;
      }
      if (a.direct) {
        float* pc = C + (int64_t)m * d.c_m + (int64_t)n * d.c_n;
        pc[0] = cr;
        pc[d.plane_c] = ci;
      } else {
        out[idx] = cr;
        out[4096 + idx] = ci;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128)
                 : "memory");
  }
}

// ------------------------------------------------------- fused mode products
// Two consecutive mode products of a degree-3 chain in one pass (the first two
// message legs of Eq. MessageTensorSelfConsistency), the intermediate kept on
// chip:
//   Y1[(o, j)][(s, n1)] = sum_(s', k) A_s'[(o, j)][k] Bt1[(s, n1)][(s', k)]
//   Y2[(o, n1)][(t, n2)] = sum_(s, j) Y1[(o, j)][(s, n1)] Bt2[(t, n2)][(s, j)]
// o the rows kept by both products, j the innermost row level of the first
// (the leg the second contracts), Bt1 / Bt2 the realified transposed messages.
// A tile is 128 rows (o, j) of the first product = 128 / chi values of o; its
// accumulator (TMEM, double-buffered) is read by the epilogue warps and
// written back, transposed to rows (o, n1) and K = (s, j), into a
// 128-byte-swizzled K-major shared-memory operand (rounded to TF32), which the
// second MMA takes with Bt2.  The second accumulator goes to global memory as
// in the streaming kernel.  Each realified message [[Re, Im], [-Im, Re]] is
// held as its three distinct chi x chi blocks (the (1,1) block equals (0,0)),
// stacked per 32-wide K chunk as rows [(0,1); (0,0); (1,0)] (t, s): the
// operand for input plane s = 1 is rows 0..2chi-1 ((0,1) over (1,1) = (0,0)),
// for s = 0 rows chi..3chi-1 ((0,0) over (1,0)), so every MMA has N = 2 chi.
//   warp 0 (one thread)  TMA: Bt1 / Bt2 blocks per site, the A ring (4 slots);
//   warp 1 (one thread)  MMA: stage 1 of each tile; stage 2 of the previous
//                        tile as soon as its operand is complete (polled
//                        while waiting for the ring), so neither waits on the
//                        other's inputs;
//   warps 2..9           two per TMEM lane quadrant, one per column half (the
//                        re / im plane): transpose into the stage-2 operand,
//                        then the output.
// The stage-2 operand has one buffer: an epilogue warp writes it for tile i
// only after it has waited for stage 2 of tile i - 1 to complete.  Every wait
// is bounded as in the streaming kernel.
constexpr int kFThreads = 320;
constexpr int kFEpi = 8;
constexpr int kFSlots = 4;
constexpr int kFStack = 3 * 64 * 128;         // one K chunk: [3 chi <= 192 rows][32 floats]
constexpr int kFBBytes = 2 * kFStack;         // chi / 32 <= 2 K chunks
constexpr int kFA2Bytes = 4 * kChunk;         // 2 chi / 32 chunks of [128][32]
constexpr int kFA2Off = 2 * kFBBytes;
constexpr int kFRingOff = kFA2Off + kFA2Bytes;
constexpr int kFBarOff = kFRingOff + kFSlots * kChunk;
constexpr int kFSmemBytes = kFBarOff + 256 + 1024;

struct FuseArgs {
  const CUtensorMap* maps;  // [3 * n_outer]: A maps, Bt1 maps, Bt2 maps
  int n_outer;
  int tiles_per_entry;
  int rank, lev0, lev1;
  int* err;
};

// row of the block stack where the N = 2 chi operand for input plane s starts
__device__ __forceinline__ int stack_row(int s, int chi) { return s == 0 ? chi : 0; }

template <int CHI>
__global__ void __launch_bounds__(kFThreads, 1) tc_chain_kernel(GemmDesc d, FuseArgs a) {
  constexpr int NR = 2 * CHI, KC = NR / 32, KCS = CHI / 32;
  constexpr uint32_t kCols = 8 * CHI;  // acc1 x 2 (2 chi each), acc2 (2 chi), padding
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sB1 = smem;
  unsigned char* sB2 = smem + kFBBytes;
  unsigned char* sA2 = smem + kFA2Off;
  unsigned char* sA = smem + kFRingOff;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kFBarOff);
  uint64_t* empty = full + kFSlots;
  uint64_t* bfull = empty + kFSlots;
  uint64_t* bempty = bfull + 1;
  uint64_t* t1full = bempty + 1;   // [2]
  uint64_t* t1empty = t1full + 2;  // [2]
  uint64_t* a2full = t1empty + 2;
  uint64_t* t2full = a2full + 1;
  uint64_t* done = t2full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int total = a.n_outer * a.tiles_per_entry;
  const int t_beg = (int)((int64_t)blockIdx.x * total / gridDim.x);
  const int t_end = (int)((int64_t)(blockIdx.x + 1) * total / gridDim.x);

  if (tid == 0) {
    for (int s = 0; s < kFSlots; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(bfull, 1);
    mbar_init(bempty, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&t1full[i], 1);
      mbar_init(&t1empty[i], kFEpi);
    }
    mbar_init(a2full, kFEpi);
    mbar_init(t2full, 1);
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const CUtensorMap* amaps = a.maps;
  const CUtensorMap* b1maps = a.maps + a.n_outer;
  const CUtensorMap* b2maps = a.maps + 2 * a.n_outer;

  if (warp == 0) {
    // ------------------------------------------------------------- producer
    if (lane == 0) {
      int it = 0, cur = -1, bl = 0;
      const uint32_t bbytes = (uint32_t)(2 * 3 * KCS * CHI * 128);
      for (int tile = t_beg; tile < t_end && !*abort_flag; ++tile) {
        const int e = tile / a.tiles_per_entry;
        if (outer_frozen(d, e)) continue;  // every role skips the same tiles
        const int mt = tile - e * a.tiles_per_entry;
        if (e != cur) {
          if (cur >= 0 && !mbar_wait(bempty, (bl - 1) & 1, a.err)) { *abort_flag = 1; break; }
          mbar_expect_tx(bfull, bbytes);
          // stack position b holds block (t, s) = (0,1), (0,0), (1,0)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const int t = b == 2 ? 1 : 0, s = b == 0 ? 1 : 0;
#pragma unroll
            for (int kk = 0; kk < KCS; ++kk) {
              const int off = kk * kFStack + b * CHI * 128;
              tma_load_2d(smem_u32(sB1 + off), b1maps + e, s * CHI + kk * 32, t * CHI, bfull);
              tma_load_2d(smem_u32(sB2 + off), b2maps + e, s * CHI + kk * 32, t * CHI, bfull);
            }
          }
          ++bl;
          cur = e;
        }
        int r = mt * 128;
        const int r0 = r % a.lev0;
        r /= a.lev0;
        const int r1 = r % a.lev1;
        const int r2 = r / a.lev1;
        bool ok = true;
#pragma unroll
        for (int c = 0; c < KC; ++c, ++it) {
          const int slot = it % kFSlots;
          if (!mbar_wait(&empty[slot], ((it / kFSlots) & 1) ^ 1, a.err)) { ok = false; break; }
          mbar_expect_tx(&full[slot], (uint32_t)kChunk);
          const int kr = c * 32, plane = kr / CHI, k = kr - plane * CHI;
          const uint32_t dst = smem_u32(sA + slot * kChunk);
          if (a.rank == 3) tma_load_3d(dst, amaps + e, k, r0, plane, &full[slot]);
          else if (a.rank == 4) tma_load_4d(dst, amaps + e, k, r0, r1, plane, &full[slot]);
          else tma_load_5d(dst, amaps + e, k, r0, r1, r2, plane, &full[slot]);
        }
        if (!ok) { *abort_flag = 1; break; }
      }
      // before the CTA exits, every copy issued has landed: slot s took the
      // loads it = s, s + kFSlots, ...
      for (int s = 0; s < kFSlots; ++s) {
        const int n = it / kFSlots + (s < it % kFSlots ? 1 : 0);
        if (n > 0) mbar_wait(&full[s], (n - 1) & 1, a.err);
      }
      if (bl > 0) mbar_wait(bfull, (bl - 1) & 1, a.err);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t idesc = make_idesc(2, 128, NR);
      const uint32_t acc2 = tmem + (uint32_t)(4 * CHI);
      int pend = -1;  // local tile whose stage 2 is not issued yet
      // stage 2 of local tile pend; its operand is complete
      auto issue2 = [&]() {
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < KC; ++c) {
          const int s = c / KCS, kk = c - s * KCS;
          const uint32_t a0 = smem_u32(sA2 + c * kChunk);
          const uint32_t b0 = smem_u32(sB2 + kk * kFStack + stack_row(s, CHI) * 128);
          // descriptors of the chunk; a 32-byte K step adds 2 to the start field
          const uint64_t da = sw128_desc(a0), db = sw128_desc(b0);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            mma_issue(0, acc2, da + 2 * ks, db + 2 * ks, idesc,
                      (c > 0 || ks > 0) ? 1u : 0u);
        }
        mma_commit(t2full);
        pend = -1;
      };
      // blocking stage 2 of the pending tile
      auto flush2 = [&]() -> bool {
        if (pend < 0) return true;
        if (!mbar_wait(a2full, pend & 1, a.err)) return false;
        issue2();
        return true;
      };
      // wait for a ring slot, issuing the pending stage 2 as soon as it is ready
      auto wait_full = [&](int slot, uint32_t par) -> bool {
        if (pend >= 0 && mbar_try_wait(a2full, pend & 1)) issue2();
        if (mbar_try_wait(&full[slot], par)) return true;
        const long long t0 = clock64();
        while (true) {
          if (pend >= 0 && mbar_try_wait(a2full, pend & 1)) issue2();
          if (mbar_try_wait(&full[slot], par)) return true;
          if (clock64() - t0 > kWaitCycles) {
            atomicOr(a.err, 2);
            return false;
          }
          __nanosleep(20);
        }
      };
      int it = 0, cur = -1, bl = 0, i = 0;  // i: tiles processed (the skipped ones not counted)
      bool ok = true;
      for (int tile = t_beg; tile < t_end && ok && !*abort_flag; ++tile) {
        const int e = tile / a.tiles_per_entry;
        if (outer_frozen(d, e)) continue;
        if (e != cur) {
          // stage 2 of the last tile of the previous entry reads its Bt2
          if (!flush2()) { ok = false; break; }
          if (cur >= 0) mma_commit(bempty);
          if (!mbar_wait(bfull, bl & 1, a.err)) { ok = false; break; }
          ++bl;
          cur = e;
        }
        const int buf = i & 1;
        if (!mbar_wait(&t1empty[buf], ((i >> 1) & 1) ^ 1, a.err)) { ok = false; break; }
        tc_fence_after();
        const uint32_t acc1 = tmem + (uint32_t)(buf * NR);
#pragma unroll
        for (int c = 0; c < KC; ++c, ++it) {
          const int slot = it % kFSlots;
          if (!wait_full(slot, (it / kFSlots) & 1)) { ok = false; break; }
          tc_fence_after();
          const int s = c / KCS, kk = c - s * KCS;
          const uint32_t a0 = smem_u32(sA + slot * kChunk);
          const uint32_t b0 = smem_u32(sB1 + kk * kFStack + stack_row(s, CHI) * 128);
          // descriptors of the chunk; a 32-byte K step adds 2 to the start field
          const uint64_t da = sw128_desc(a0), db = sw128_desc(b0);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            mma_issue(0, acc1, da + 2 * ks, db + 2 * ks, idesc,
                      (c > 0 || ks > 0) ? 1u : 0u);
          mma_commit(&empty[slot]);
        }
        if (!ok) break;
        mma_commit(&t1full[buf]);
        // at most one stage 2 outstanding: the previous tile's goes first
        if (!flush2()) { ok = false; break; }
        pend = i;
        ++i;
      }
      if (ok && !*abort_flag) ok = flush2();
      if (!ok) *abort_flag = 1;
      mma_commit(done);
      mbar_wait(done, 0, a.err);
    }
    __syncwarp();
  } else {
    // ----------------------------------------------- transpose and epilogue
    const int q = warp & 3;              // TMEM lane quadrant
    const int h = (warp - 2) >> 2;       // column half: plane s of Y1, t of Y2
    const int row = q * 32 + lane;       // (g, j) of stage 1, (g, n1) of stage 2
    const int g = row / CHI, j = row - g * CHI;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    // the stage-2 operand: K index (s = h, j) -> chunk h * CHI / 32 + j / 32,
    // column j % 32 = lane; row g * CHI + n1; the 16-byte unit of a row r is
    // swizzled by r % 8 = n1 % 8
    unsigned char* a2base = sA2 + (h * KCS + j / 32) * kChunk + (g * CHI) * 128 + ((lane & 3) << 2);
    uint32_t uoff[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) uoff[u] = (uint32_t)((((lane >> 2) ^ u)) << 4);
    int i = 0;  // tiles processed (the skipped ones not counted)
    for (int tile = t_beg; tile < t_end; ++tile) {
      if (*abort_flag) break;
      const int e = tile / a.tiles_per_entry;
      if (outer_frozen(d, e)) continue;
      const int mt = tile - e * a.tiles_per_entry;
      const int buf = i & 1;
      if (!mbar_wait(&t1full[buf], (i >> 1) & 1, a.err)) { *abort_flag = 1; break; }
      tc_fence_after();
      __syncwarp();
#pragma unroll
      for (int cc = 0; cc < KCS; ++cc) {
        float v[32];
        tmem_ld32(lane_base + (uint32_t)(buf * NR + h * CHI + cc * 32), v);
        unsigned char* rb = a2base + cc * 32 * 128;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj)
          *reinterpret_cast<uint32_t*>(rb + jj * 128 + uoff[jj & 7]) = to_tf32(v[jj]);
      }
      tc_fence_before();
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&t1empty[buf]);
        mbar_arrive(a2full);
      }
      if (!mbar_wait(t2full, i & 1, a.err)) { *abort_flag = 1; break; }
      tc_fence_after();
      __syncwarp();
      float* C = d.C[e] + ROW_C(d, mt * 128 + row) + (h ? d.plane_c : 0);
#pragma unroll
      for (int cc = 0; cc < KCS; ++cc) {
        float v[32];
        tmem_ld32(lane_base + (uint32_t)(4 * CHI + h * CHI + cc * 32), v);
        float* Cc = C + cc * 32 * CHI;  // columns n2 = cc * 32 + jj at stride CHI
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) Cc[jj * CHI] = v[jj];
      }
      tc_fence_before();
      __syncwarp();
      ++i;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                 : "memory");
  }
}

// Self-test of the bounded device wait: one thread waits on an mbarrier that
// nothing arrives at, through the same mbar_wait every tcgen05 kernel here
// uses.  The wait must give up after its limit (about one second), set bit 1
// of *err and return, leaving the context usable.
__global__ void wait_selftest_kernel(int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && mbar_wait(&bar, 0, err)) atomicOr(err, 4);  // 4: the wait did not give up
  __syncthreads();
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Row levels of the descriptor's A operand, innermost first, adjacent levels
// merged where they are contiguous, then boxed into 128-row tiles.
struct Levels {
  int n = 0;
  int64_t size[3], stride[3];
  int box[3];
};

bool row_levels(const GemmDesc& d, Levels* L) {
  int64_t sz[3], st[3];
  int n = 0;
  if (d.M3 > 1) {
    if (d.M % (d.M2 * d.M3)) return false;
    sz[0] = d.M3; st[0] = d.a_m3; sz[1] = d.M2; st[1] = d.a_m2; sz[2] = d.M / (d.M2 * d.M3);
    st[2] = d.a_m; n = 3;
  } else if (d.M2 > 1) {
    if (d.M % d.M2) return false;
    sz[0] = d.M2; st[0] = d.a_m2; sz[1] = d.M / d.M2; st[1] = d.a_m; n = 2;
  } else {
    sz[0] = d.M; st[0] = d.a_m; n = 1;
  }
  // drop unit levels, merge contiguous neighbours
  int m = 0;
  for (int i = 0; i < n; ++i) {
    if (sz[i] == 1) continue;
    if (m > 0 && st[i] == L->size[m - 1] * L->stride[m - 1]) {
      L->size[m - 1] *= sz[i];
      continue;
    }
    L->size[m] = sz[i];
    L->stride[m] = st[i];
    ++m;
  }
  if (m == 0) { L->size[0] = 1; L->stride[0] = d.a_m; m = 1; }
  L->n = m;
  int64_t rem = 128;
  for (int i = 0; i < m; ++i) {
    if (rem == 1) { L->box[i] = 1; continue; }
    if (L->size[i] >= rem) {
      if (L->size[i] % rem) return false;
      L->box[i] = (int)rem;
      rem = 1;
    } else {
      if (rem % L->size[i]) return false;
      L->box[i] = (int)L->size[i];
      rem /= L->size[i];
    }
  }
  return rem == 1;
}

int g_num_sms = 0;

}  // namespace

bool tc_stream_encode(const GemmDesc& d, const float* const* A, const float* const* B, int n_outer,
                      void* host_maps, TcStreamPlan* p) {
  const int chi = d.N;
  if (d.prec != TN_TF32 || !d.b_pre || d.K1 != 1 || d.K2 != chi || d.a_k2 != 1 || d.conj_a ||
      d.accumulate || d.n_inner != 1 || (chi != 32 && chi != 64) || d.M % 128 != 0 ||
      n_outer < 1)
    return false;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  Levels L;
  if (!row_levels(d, &L)) return false;
  const int rank = L.n + 2;
  if (rank > 5) return false;
  for (int i = 0; i < L.n; ++i)
    if ((L.stride[i] * 4) % 16 || L.stride[i] * 4 >= (int64_t(1) << 40)) return false;
  if ((d.plane_a * 4) % 16) return false;
  if (d.c_n == 1 && (d.c_m % 4 || (d.M2 > 1 && d.c_m2 % 4) || (d.M3 > 1 && d.c_m3 % 4) ||
                     d.plane_c % 4))
    return false;
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(host_maps);
  for (int e = 0; e < n_outer; ++e) {
    if ((reinterpret_cast<uintptr_t>(A[e]) & 15) || (reinterpret_cast<uintptr_t>(B[e]) & 15))
      return false;
    cuuint64_t dims[5], strides[4];
    cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
    dims[0] = (cuuint64_t)chi;
    box[0] = 32;
    for (int i = 0; i < L.n; ++i) {
      dims[1 + i] = (cuuint64_t)L.size[i];
      strides[i] = (cuuint64_t)(L.stride[i] * 4);
      box[1 + i] = (cuuint32_t)L.box[i];
    }
    dims[rank - 1] = 2;
    strides[rank - 2] = (cuuint64_t)(d.plane_a * 4);
    box[rank - 1] = 1;
    if (enc(&maps[e], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank,
            const_cast<float*>(A[e]), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
    // Bt: real [2 chi][2 chi] row-major
    cuuint64_t bd[2] = {(cuuint64_t)(2 * chi), (cuuint64_t)(2 * chi)};
    cuuint64_t bs[1] = {(cuuint64_t)(2 * chi * 4)};
    cuuint32_t bb[2] = {32, (cuuint32_t)(2 * chi)};
    if (enc(&maps[n_outer + e], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(B[e]), bd,
            bs, bb, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  p->rank = rank;
  p->lev0 = (int)(L.n > 0 ? L.size[0] : 1);
  p->lev1 = (int)(L.n > 1 ? L.size[1] : 1);
  if (rank == 3) p->lev0 = (int)L.size[0];
  p->n_outer = n_outer;
  return true;
}

size_t tc_stream_map_bytes(int n_outer) { return (size_t)2 * n_outer * sizeof(CUtensorMap); }

cudaError_t tc_stream_prepare() {
  static std::once_flag once;
  static cudaError_t result = cudaSuccess;
  std::call_once(once, [] {
    result = cudaFuncSetAttribute(tc_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kSmemBytes);
    if (result == cudaSuccess)
      result = cudaFuncSetAttribute(tc_chain_kernel<32>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kFSmemBytes);
    if (result == cudaSuccess)
      result = cudaFuncSetAttribute(tc_chain_kernel<64>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kFSmemBytes);
    if (result == cudaSuccess)
      result = cudaFuncSetAttribute(tc_close_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kCSmemBytes);
    if (result == cudaSuccess)
      result = cudaFuncSetAttribute(tc_close_kernel,
                                    cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int dev = 0, sms = 0;
    if (result == cudaSuccess) result = cudaGetDevice(&dev);
    if (result == cudaSuccess)
      result = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (result == cudaSuccess) g_num_sms = sms;
  });
  return result;
}

cudaError_t launch_tc_stream(const GemmDesc& d, const TcStreamPlan& p, int* err, cudaStream_t st) {
  cudaError_t e = tc_stream_prepare();
  if (e != cudaSuccess) return e;
  StreamArgs a;
  a.maps = reinterpret_cast<const CUtensorMap*>(p.maps);
  a.n_outer = p.n_outer;
  a.tiles_per_entry = d.M / 128;
  a.chi = d.N;
  a.nr = 2 * d.N;
  a.kc = 2 * d.N / 32;
  a.rank = p.rank;
  a.lev0 = p.lev0;
  a.lev1 = p.lev1;
  a.err = err;
  const int total = a.n_outer * a.tiles_per_entry;
  const int grid = total < g_num_sms ? total : g_num_sms;
  tc_stream_kernel<<<grid, kThreads, kSmemBytes, st>>>(d, a);
  return cudaGetLastError();
}


bool tc_close_encode(const GemmDesc& d, const float* const* A, const float* const* B, int n_outer,
                     size_t part_floats, void* host_maps, TcStreamPlan* p) {
  if (d.prec != TN_TF32 || d.b_pre || d.M != 64 || d.N != 64 || d.a_k2 != 1 || d.b_k2 != 1 ||
      d.n_inner < 1 || d.K2 % 32 || d.M2 > 1 || d.M3 > 1 || d.accumulate || n_outer < 1)
    return false;
  // entries (outer, inner) in the order the partial buffer and the reduce use
  const int n_ent = n_outer * d.n_inner;
  if (tc_stream_prepare() != cudaSuccess) return false;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const int64_t s_a[3] = {d.a_m, d.K1 > 1 ? d.a_k1 : d.plane_a, d.plane_a};
  const int64_t s_b[3] = {d.b_n, d.K1 > 1 ? d.b_k1 : d.plane_b, d.plane_b};
  for (int i = 0; i < 3; ++i)
    if (s_a[i] <= 0 || s_b[i] <= 0 || (s_a[i] * 4) % 16 || (s_b[i] * 4) % 16) return false;
  const int chunks = d.K1 * d.K2 / 32;
  int S = 1;
  while ((int64_t)n_ent * S * 2 <= 2LL * g_num_sms && chunks / (S * 2) >= 4) S *= 2;
  const int per = (chunks + S - 1) / S;
  S = (chunks + per - 1) / per;  // every split holds at least one chunk
  if ((size_t)S * n_ent * 2 * 4096 > part_floats) return false;
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(host_maps);
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const cuuint32_t box[4] = {32, 64, 1, 2};
  if ((d.a_in * 4) % 16 || (d.b_in * 4) % 16) return false;
  for (int e = 0; e < n_ent; ++e) {
    const int o = e / d.n_inner, in = e - o * d.n_inner;
    const float* Ae = A[o] + (int64_t)in * d.a_in;
    const float* Be = B[o] + (int64_t)in * d.b_in;
    if ((reinterpret_cast<uintptr_t>(Ae) & 15) || (reinterpret_cast<uintptr_t>(Be) & 15))
      return false;
    cuuint64_t dims[4] = {(cuuint64_t)d.K2, 64, (cuuint64_t)d.K1, 2};
    cuuint64_t sa[3] = {(cuuint64_t)(s_a[0] * 4), (cuuint64_t)(s_a[1] * 4),
                        (cuuint64_t)(s_a[2] * 4)};
    cuuint64_t sb[3] = {(cuuint64_t)(s_b[0] * 4), (cuuint64_t)(s_b[1] * 4),
                        (cuuint64_t)(s_b[2] * 4)};
    if (enc(&maps[e], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(Ae), dims, sa, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
    if (enc(&maps[n_ent + e], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(Be), dims,
            sb, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  p->kind = 1;
  p->n_outer = n_ent;  // entries: outer x inner
  p->splits = S;
  p->rank = 4;
  return true;
}

cudaError_t launch_tc_close(const GemmDesc& d, const TcStreamPlan& p, float* part, int* err,
                            cudaStream_t st) {
  {
    cudaError_t e = tc_stream_prepare();
    if (e != cudaSuccess) return e;
  }
  CloseArgs a;
  a.maps = reinterpret_cast<const CUtensorMap*>(p.maps);
  a.n_outer = p.n_outer;
  a.chunks = d.K1 * d.K2 / 32;
  a.per_split = (a.chunks + p.splits - 1) / p.splits;
  a.K2 = d.K2;
  a.direct = p.splits == 1 ? 1 : 0;
  a.part = part;
  a.err = err;
  dim3 grid(p.splits, p.n_outer);
  tc_close_kernel<<<grid, kCThreads, kCSmemBytes, st>>>(d, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || a.direct) return e;
  return launch_tc_reduce(d, part, p.splits, st);
}


// The second product reads exactly what the first writes, with the first's
// innermost row level as its contracted index: for every row (o, j) and
// column n1 of the first, element (o, n1; k = j) of the second.  Checked
// element by element; the result depends only on the two descriptors'
// strides, so it is kept per distinct pair.
bool chain_layouts_match(const GemmDesc& d1, const GemmDesc& d2) {
  const int chi = d1.N;
  const int64_t key[] = {d1.M,   d1.N,   d1.M2,   d1.M3,   d1.c_m,  d1.c_m2, d1.c_m3,
                         d1.c_n, d2.M2,  d2.M3,   d2.a_m,  d2.a_m2, d2.a_m3, d2.a_k2};
  constexpr int nk = (int)(sizeof(key) / sizeof(key[0]));
  static std::mutex mu;
  static std::vector<std::pair<std::vector<int64_t>, bool>> cache;
  std::vector<int64_t> kv(key, key + nk);
  {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& c : cache)
      if (c.first == kv) return c.second;
  }
  bool ok = true;
  for (int m1 = 0; m1 < d1.M && ok; ++m1) {
    const int o = m1 / chi, j = m1 - o * chi;
    for (int n1 = 0; n1 < chi; ++n1) {
      const int64_t w = ROW_C(d1, m1) + (int64_t)n1 * d1.c_n;
      const int64_t r = ROW_A(d2, o * chi + n1) + (int64_t)j * d2.a_k2;
      if (w != r) { ok = false; break; }
    }
  }
  std::lock_guard<std::mutex> lk(mu);
  cache.emplace_back(kv, ok);
  return ok;
}

bool tc_chain_encode(const GemmDesc& d1, const GemmDesc& d2, const float* const* A,
                     const float* const* B1, const float* const* A2, const float* const* B2,
                     float* const* C1, int n_outer, void* host_maps, TcStreamPlan* p) {
  const int chi = d1.N;
  auto mode_ok = [&](const GemmDesc& d) {
    return d.prec == TN_TF32 && d.b_pre && d.K1 == 1 && d.K2 == chi && d.N == chi && !d.conj_a &&
           !d.accumulate && d.n_inner == 1 && d.M == d1.M;
  };
  if (!mode_ok(d1) || !mode_ok(d2) || d1.a_k2 != 1 || (chi != 32 && chi != 64) ||
      d1.M % 128 != 0 || n_outer < 1 || d1.plane_c != d2.plane_a || d2.c_n != chi)
    return false;
  if (!chain_layouts_match(d1, d2)) return false;
  for (int e = 0; e < n_outer; ++e)
    if (A2[e] != C1[e] || (reinterpret_cast<uintptr_t>(B2[e]) & 15)) return false;
  if (tc_stream_prepare() != cudaSuccess) return false;
  // the A and Bt1 maps as for the streaming kernel, with chi-row Bt boxes
  std::vector<unsigned char> tmp(tc_stream_map_bytes(n_outer) + 64);
  unsigned char* t2 = (unsigned char*)(((uintptr_t)tmp.data() + 63) & ~uintptr_t(63));
  TcStreamPlan sp;
  if (!tc_stream_encode(d1, A, B1, n_outer, t2, &sp)) return false;
  EncodeTiledFn enc = encode_fn();
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(host_maps);
  const CUtensorMap* src = reinterpret_cast<const CUtensorMap*>(t2);
  const cuuint32_t estr[2] = {1, 1};
  const cuuint64_t bd[2] = {(cuuint64_t)(2 * chi), (cuuint64_t)(2 * chi)};
  const cuuint64_t bs[1] = {(cuuint64_t)(2 * chi * 4)};
  const cuuint32_t bb[2] = {32, (cuuint32_t)chi};
  for (int e = 0; e < n_outer; ++e) {
    maps[e] = src[e];
    if (enc(&maps[n_outer + e], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(B1[e]),
            bd, bs, bb, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
    if (enc(&maps[2 * n_outer + e], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
            const_cast<float*>(B2[e]), bd, bs, bb, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  *p = sp;
  p->kind = 2;
  return true;
}

size_t tc_chain_map_bytes(int n_outer) { return (size_t)3 * n_outer * sizeof(CUtensorMap); }

cudaError_t launch_tc_chain(const GemmDesc& d1, const GemmDesc& d2, const TcStreamPlan& p,
                            int* err, cudaStream_t st) {
  cudaError_t e = tc_stream_prepare();
  if (e != cudaSuccess) return e;
  FuseArgs a;
  a.maps = reinterpret_cast<const CUtensorMap*>(p.maps);
  a.n_outer = p.n_outer;
  a.tiles_per_entry = d1.M / 128;
  a.rank = p.rank;
  a.lev0 = p.lev0;
  a.lev1 = p.lev1;
  a.err = err;
  const int total = a.n_outer * a.tiles_per_entry;
  const int grid = total < g_num_sms ? total : g_num_sms;
  if (d1.N == 64) tc_chain_kernel<64><<<grid, kFThreads, kFSmemBytes, st>>>(d2, a);
  else tc_chain_kernel<32><<<grid, kFThreads, kFSmemBytes, st>>>(d2, a);
  return cudaGetLastError();
}


cudaError_t launch_wait_selftest(int* err, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(err);
  return cudaGetLastError();
}

}  // namespace tnbp
