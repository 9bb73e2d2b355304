// Tensor-core (tcgen05, sm_103a) batched complex GEMM for the message and gate
// contractions (TF32 / BF16 inputs, FP32 accumulation in tensor memory).
//
// A complex product C = op(A) op(B) on planar data becomes one real GEMM
// D[mr][nr] = sum_kr Ar[mr][kr] Br[nr][kr], in one of two forms:
//   REAL_B (mode products, leg matrices: many rows, K and N = chi):
//     mr = m, nr = (t, n), kr = (s, k):  Ar = [A_re | A_im],
//     Br[(t,n)][(s,k)] = [[B_re, B_im], [-B_im, B_re]][s][t] (realified B), so
//     D[m][(0,n)] = C_re, D[m][(1,n)] = C_im;
//   QUAD (closes: K = chi^2 .. 2 chi^2, M = N = chi):
//     mr = (s, m), nr = (t, n), kr = k:  D = P[(s,m)][(t,n)] = sum_k A_s[m][k] B_t[k][n],
//     and the epilogue forms C_re = P_rr - sa sb P_ii, C_im = sb P_ri + sa P_ir
//     (sa, sb = -1 for a conjugated operand); K may be split over CTAs, the
//     partial products reduced by a second kernel in a fixed order.
// The arithmetic is 4 real multiply-adds per complex one in both forms.
//
// CTA: 256 threads.  Warps 4..7 stage operand tiles: they read the strided
// source through the same descriptor as the CUDA-core kernel (consecutive
// threads walk the operand's contiguous index) and write K-major 128-byte
// swizzled rows (32 x 4-byte or 64 x 2-byte elements per row, 8-row atoms of
// 1024 bytes), 3 stages, each closed by an mbarrier.  One thread of warp 0
// issues tcgen05.mma (M = 128, N = 16..128, K = 8 TF32 / 16 BF16 per
// instruction) into a 128-column TMEM accumulator and releases each stage with
// tcgen05.commit; warps 0..3 read the accumulator back with tcgen05.ld (one
// 32-lane quadrant each) and store C.  Every mbarrier wait is bounded (about
// one second of clock64 time): on expiry the kernel sets bit 1 of *err, stops
// issuing, still waits (bounded) for its own issued MMAs and frees TMEM.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "tc_common.cuh"
#include "tnbp.h"

namespace tnbp {
namespace {

using namespace tc;

constexpr int kTM = 128;          // tile rows (MMA M)
constexpr int kTN = 128;          // max tile columns (MMA N)
constexpr int kRowBytes = 128;    // one K tile = one swizzled 128-byte row per M/N row
constexpr int kStages = 3;
constexpr int kThreads = 256;
constexpr int kTmemCols = 128;
constexpr int kBatch = 8;                        // 16-byte loads in flight per producer thread

struct TcSmem {
  static constexpr int kA = kTM * kRowBytes;   // 16 KB per stage
  static constexpr int kB = kTN * kRowBytes;   // 16 KB per stage
  // the hi tiles of every stage; with split precision the lo tiles follow
  static constexpr int kHi = kStages * (kA + kB);
  __host__ __device__ static constexpr int bar_off(int x3) { return kHi * (x3 ? 2 : 1); }
  __host__ __device__ static constexpr int bytes(int x3) { return bar_off(x3) + 128; }
};

__device__ __forceinline__ int64_t koff(int k, int K2, int64_t s1, int64_t s2) {
  const int k1 = k / K2;
  return (int64_t)k1 * s1 + (int64_t)(k - k1 * K2) * s2;
}

struct TcArgs {
  int quad;        // 0: REAL_B, 1: QUAD
  int bf16;        // operand format: 0 TF32, 1 BF16
  int x3;          // split precision: x = hi + lo, D += A_hi B_hi + A_hi B_lo + A_lo B_hi
  int mr, nr, kr;  // real GEMM sizes
  int tn;          // N tile (multiple of 16, <= 128)
  int splits;      // K splits
  int k_per_split; // real K per split (multiple of the K tile)
  float* part;     // partial outputs [split][outer][inner][2][M][N] (splits > 1)
  int* err;
};

// element (mr, kr) of the real A operand
__device__ __forceinline__ float load_a(const GemmDesc& d, const TcArgs& t, const float* A, int mr,
                                        int kr) {
  const int K = d.K1 * d.K2;
  int m, k, s;
  if (t.quad) { s = mr >= d.M; m = mr - s * d.M; k = kr; }
  else { s = kr >= K; k = kr - s * K; m = mr; }
  const int64_t off =
      ROW_A(d, m) + koff(k, d.K2, d.a_k1, d.a_k2) + (s ? d.plane_a : 0);
  float v = __ldg(A + off);
  if (!t.quad && s && d.conj_a) v = -v;
  return v;
}

// element (nr, kr) of the real B operand (stored N x K)
__device__ __forceinline__ float load_b(const GemmDesc& d, const TcArgs& t, const float* B, int nr,
                                        int kr) {
  const int K = d.K1 * d.K2;
  const int tt = nr >= d.N;
  const int n = nr - tt * d.N;
  if (t.quad) {
    const int64_t off = (int64_t)n * d.b_n + koff(kr, d.K2, d.b_k1, d.b_k2) + (tt ? d.plane_b : 0);
    return __ldg(B + off);
  }
  const int s = kr >= K;
  const int k = kr - s * K;
  const int64_t base = (int64_t)n * d.b_n + koff(k, d.K2, d.b_k1, d.b_k2);
  if (s == tt) return __ldg(B + base);                       // B_re on the diagonal blocks
  float bi = __ldg(B + base + d.plane_b);                    // B_im off the diagonal
  if (d.conj_b) bi = -bi;
  return s == 0 ? bi : -bi;
}

// Four consecutive K elements of one row as one 16-byte (TF32) or 8-byte (BF16) store.
__device__ __forceinline__ void store_k4(unsigned char* tile, int row, int kk, float4 v, int bf16) {
  if (bf16) {
    const int chunk = (kk >> 3) ^ (row & 7);
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t*>(&lo);
    u.y = *reinterpret_cast<uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(tile + row * kRowBytes + chunk * 16 + (kk & 7) * 2) = u;
  } else {
    const int chunk = (kk >> 2) ^ (row & 7);
    uint4 u = make_uint4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
    *reinterpret_cast<uint4*>(tile + row * kRowBytes + chunk * 16) = u;
  }
}

// The part of v that the operand format does not hold: v - round(v).
__device__ __forceinline__ float lo_part(float v, int bf16) {
  const float hi = bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : __uint_as_float(to_tf32(v));
  return v - hi;
}
__device__ __forceinline__ float4 lo_part4(float4 v, int bf16) {
  return make_float4(lo_part(v.x, bf16), lo_part(v.y, bf16), lo_part(v.z, bf16), lo_part(v.w, bf16));
}

__device__ __forceinline__ void store_elem(unsigned char* tile, int row, int kk, float v, int bf16) {
  if (bf16) {
    // 64 bf16 per 128-byte row; 16-byte chunk = 8 elements
    const int chunk = (kk >> 3) ^ (row & 7);
    __nv_bfloat16* p = reinterpret_cast<__nv_bfloat16*>(tile + row * kRowBytes + chunk * 16) + (kk & 7);
    *p = __float2bfloat16_rn(v);
  } else {
    const int chunk = (kk >> 2) ^ (row & 7);
    uint32_t* p = reinterpret_cast<uint32_t*>(tile + row * kRowBytes + chunk * 16) + (kk & 3);
    *p = to_tf32(v);
  }
}

__global__ void __launch_bounds__(kThreads, 2) tc_gemm_kernel(GemmDesc d, TcArgs t) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // align the dynamic buffer to 1024 bytes (swizzle atoms)
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = smem;
  unsigned char* sB = smem + kStages * TcSmem::kA;
  unsigned char* sAl = smem + TcSmem::kHi;  // lo tiles (split precision only)
  unsigned char* sBl = sAl + kStages * TcSmem::kA;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + TcSmem::bar_off(t.x3));
  uint64_t* empty = full + kStages;
  uint64_t* accum = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int z = blockIdx.z;
  const int split = z % t.splits;
  z /= t.splits;
  const int outer = z / d.n_inner, inner = z - (z / d.n_inner) * d.n_inner;
  // a converged component of a union: nothing is initialised yet, the whole
  // CTA leaves together
  if (outer_frozen(d, outer)) return;
  const float* A = d.A[outer] + inner * d.a_in;
  const float* B = d.B[outer] + inner * d.b_in;
  const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * t.tn;
  const int kbeg = split * t.k_per_split;
  const int kend = min(t.kr, kbeg + t.k_per_split);
  const int kelems = t.bf16 ? 64 : 32;  // K elements per 128-byte row
  const int ntiles = (kend - kbeg + kelems - 1) / kelems;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 128);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp >= 4) {
    // ---------------------------------------------------------- producers
    const int pt = tid - 128;
    const int K = d.K1 * d.K2;
    // Vector paths: 16-byte loads along K (each 4 x 4-byte chunk of a K tile lies
    // inside one K2 run and one plane) or along M / N (4 consecutive rows).
    const bool kvec = (d.K2 % kelems == 0) && (K % kelems == 0) && (kbeg % kelems == 0) &&
                      (t.kr % kelems == 0);
    const bool a_kvec = kvec && d.a_k2 == 1 && (d.a_m % 4 == 0) && (d.a_k1 % 4 == 0) &&
                        (d.plane_a % 4 == 0) && (d.a_in % 4 == 0) &&
                        (d.M2 <= 1 || d.a_m2 % 4 == 0) && (d.M3 <= 1 || d.a_m3 % 4 == 0);
    // A rows contiguous: four consecutive rows m..m+3 (same upper row levels, same
    // plane) are adjacent
    bool a_rows4;
    if (d.M3 > 1) a_rows4 = d.a_m3 == 1 && d.M3 % 4 == 0 && d.a_m % 4 == 0 && d.a_m2 % 4 == 0;
    else if (d.M2 > 1) a_rows4 = d.a_m2 == 1 && d.M2 % 4 == 0 && d.a_m % 4 == 0;
    else a_rows4 = d.a_m == 1;
    const bool a_mvec = !a_kvec && (d.M % 4 == 0) && (d.a_k1 % 4 == 0) && (d.a_k2 % 4 == 0) &&
                        (d.plane_a % 4 == 0) && (d.a_in % 4 == 0) && a_rows4;
    // B K-contiguous: the closes' long operand, or the realified transposed small
    // operand of a b_pre descriptor (read as a plain real matrix, no signs)
    const bool b_kvec = kvec && d.b_k2 == 1 && (d.b_n % 4 == 0) && (d.b_k1 % 4 == 0) &&
                        (d.plane_b % 4 == 0) && (d.b_in % 4 == 0) && (t.quad || d.b_pre);
    const bool b_nvec = !b_kvec && d.b_n == 1 && (d.N % 4 == 0) && (d.b_k1 % 4 == 0) &&
                        (d.b_k2 % 4 == 0) && (d.plane_b % 4 == 0) && (d.b_in % 4 == 0) &&
                        (t.tn % 4 == 0) && (n0 % 4 == 0);
    const bool a_kfast = d.a_k2 == 1 && !(d.M2 > 1 && d.M3 <= 1 && d.a_m2 == 1) &&
                         !(d.M3 > 1 && d.a_m3 == 1);
    const bool a_async = !t.bf16 && !t.x3 && a_kvec && ((reinterpret_cast<uintptr_t>(A) & 15) == 0) &&
                         !(d.conj_a && !t.quad);
    const bool b_async = !t.bf16 && !t.x3 && b_kvec && ((reinterpret_cast<uintptr_t>(B) & 15) == 0);
    const bool b_nfast = d.b_n == 1;
    const bool aligned = ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) == 0;
    for (int kt = 0; kt < ntiles; ++kt) {
      const int s = kt % kStages;
      const uint32_t par = ((kt / kStages) & 1) ^ 1;
      if (!mbar_wait(&empty[s], par, t.err)) { *abort_flag = 1; }
      if (*abort_flag) { mbar_arrive(&full[s]); continue; }
      unsigned char* ta = sA + s * TcSmem::kA;
      unsigned char* tb = sB + s * TcSmem::kB;
      unsigned char* tal = sAl + s * TcSmem::kA;
      unsigned char* tbl = sBl + s * TcSmem::kB;
      const int k0 = kbeg + kt * kelems;
      // TF32 operands whose K index is contiguous are copied with cp.async
      // straight into their swizzled place (the tensor core reads the FP32 bits
      // as TF32); the stage's mbarrier then completes when the copies land, so
      // the producers run ahead by up to kStages stages.  Other operands go
      // through registers: kBatch 16-byte loads in flight per thread, then
      // conversion and stores.
      if (a_async) {
        int sa, kloc;
        if (t.quad) { sa = 0; kloc = k0; } else { sa = k0 >= K; kloc = k0 - sa * K; }
        const int64_t kbase = koff(kloc, d.K2, d.a_k1, d.a_k2);
        const uint32_t base_s = smem_u32(ta);
        for (int c = pt; c < kTM * 8; c += 128) {
          const int row = c >> 3, q = c & 7;
          const int mr = m0 + row;
          const bool ok = mr < t.mr && k0 + q * 4 < kend;
          const float* src = A;
          if (ok) {
            int m = mr, splane = sa;
            if (t.quad) { splane = mr >= d.M; m = mr - splane * d.M; }
            src = A + ROW_A(d, m) + kbase + q * 4 + (splane ? d.plane_a : 0);
          }
          cp_async16(base_s + row * kRowBytes + ((q ^ (row & 7)) << 4), src, ok);
        }
      } else if (a_kvec && aligned) {
        // A: K-contiguous; the whole tile lies in one plane (s) and one K2 run
        int sa, kloc;
        if (t.quad) { sa = 0; kloc = k0; } else { sa = k0 >= K; kloc = k0 - sa * K; }
        const int64_t kbase = koff(kloc, d.K2, d.a_k1, d.a_k2);
        const int qpr = kelems / 4, total = kTM * qpr;
        for (int base = 0; base < total; base += 128 * kBatch) {
          float4 v[kBatch];
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int c = base + u * 128 + pt;
            const int row = c / qpr, q = c - (c / qpr) * qpr;
            const int mr = m0 + row;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c < total && mr < t.mr && k0 + q * 4 < kend) {
              int m = mr, splane = sa;
              if (t.quad) { splane = mr >= d.M; m = mr - splane * d.M; }
              v[u] = __ldg(reinterpret_cast<const float4*>(A + ROW_A(d, m) +
                                                           kbase + q * 4 + (splane ? d.plane_a : 0)));
              if (!t.quad && splane && d.conj_a) {
                v[u].x = -v[u].x; v[u].y = -v[u].y; v[u].z = -v[u].z; v[u].w = -v[u].w;
              }
            }
          }
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int c = base + u * 128 + pt;
            if (c < total) {
              const int row = c / qpr, kk = (c - (c / qpr) * qpr) * 4;
              store_k4(ta, row, kk, v[u], t.bf16);
              if (t.x3) store_k4(tal, row, kk, lo_part4(v[u], t.bf16), t.bf16);
            }
          }
        }
      } else if (a_mvec && aligned) {
        const int total = (kTM / 4) * kelems;
        for (int base = 0; base < total; base += 128 * kBatch) {
          float4 v[kBatch];
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int c = base + u * 128 + pt;
            const int rq = c % (kTM / 4), kk = c / (kTM / 4);
            const int mr = m0 + rq * 4, kr = k0 + kk;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c < total && mr < t.mr && kr < kend) {
              int sp, m, k;
              if (t.quad) { sp = mr >= d.M; m = mr - sp * d.M; k = kr; }
              else { sp = kr >= K; k = kr - sp * K; m = mr; }
              v[u] = __ldg(reinterpret_cast<const float4*>(
                  A + ROW_A(d, m) + koff(k, d.K2, d.a_k1, d.a_k2) +
                  (sp ? d.plane_a : 0)));
              if (!t.quad && sp && d.conj_a) {
                v[u].x = -v[u].x; v[u].y = -v[u].y; v[u].z = -v[u].z; v[u].w = -v[u].w;
              }
            }
          }
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int c = base + u * 128 + pt;
            if (c >= total) continue;
            const int row = (c % (kTM / 4)) * 4, kk = c / (kTM / 4);
            store_elem(ta, row, kk, v[u].x, t.bf16);
            store_elem(ta, row + 1, kk, v[u].y, t.bf16);
            store_elem(ta, row + 2, kk, v[u].z, t.bf16);
            store_elem(ta, row + 3, kk, v[u].w, t.bf16);
            if (t.x3) {
              const float4 l = lo_part4(v[u], t.bf16);
              store_elem(tal, row, kk, l.x, t.bf16);
              store_elem(tal, row + 1, kk, l.y, t.bf16);
              store_elem(tal, row + 2, kk, l.z, t.bf16);
              store_elem(tal, row + 3, kk, l.w, t.bf16);
            }
          }
        }
      } else {
        for (int i = pt; i < kTM * kelems; i += 128) {
          int row, kk;
          if (a_kfast) { kk = i % kelems; row = i / kelems; }
          else { row = i % kTM; kk = i / kTM; }
          const int mr = m0 + row, kr = k0 + kk;
          const float v = (mr < t.mr && kr < kend) ? load_a(d, t, A, mr, kr) : 0.f;
          store_elem(ta, row, kk, v, t.bf16);
          if (t.x3) store_elem(tal, row, kk, lo_part(v, t.bf16), t.bf16);
        }
      }
      if (b_async) {
        const int64_t kbase = koff(k0, d.K2, d.b_k1, d.b_k2);
        const uint32_t base_s = smem_u32(tb);
        for (int c = pt; c < t.tn * 8; c += 128) {
          const int row = c >> 3, q = c & 7;
          const int nr = n0 + row;
          const bool ok = nr < t.nr && k0 + q * 4 < kend;
          const float* src = B;
          if (ok) {
            const int tt = nr >= d.N;
            const int n = nr - tt * d.N;
            src = B + (int64_t)n * d.b_n + kbase + q * 4 + (tt ? d.plane_b : 0);
          }
          cp_async16(base_s + row * kRowBytes + ((q ^ (row & 7)) << 4), src, ok);
        }
      } else if (b_kvec && aligned) {
        const int64_t kbase = koff(k0, d.K2, d.b_k1, d.b_k2);
        const int qpr = kelems / 4, total = t.tn * qpr;
        for (int base = 0; base < total; base += 128 * kBatch) {
          float4 v[kBatch];
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int c = base + u * 128 + pt;
            const int row = c / qpr, q = c - (c / qpr) * qpr;
            const int nr = n0 + row;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c < total && nr < t.nr && k0 + q * 4 < kend) {
              const int tt = nr >= d.N;
              const int n = nr - tt * d.N;
              v[u] = __ldg(reinterpret_cast<const float4*>(B + (int64_t)n * d.b_n + kbase + q * 4 +
                                                           (tt ? d.plane_b : 0)));
            }
          }
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int c = base + u * 128 + pt;
            if (c < total) {
              const int row = c / qpr, kk = (c - (c / qpr) * qpr) * 4;
              store_k4(tb, row, kk, v[u], t.bf16);
              if (t.x3) store_k4(tbl, row, kk, lo_part4(v[u], t.bf16), t.bf16);
            }
          }
        }
      } else if (b_nvec && aligned) {
        // B: N-contiguous; four consecutive rows nr share (t, s, k)
        const int total = (t.tn / 4) * kelems;
        for (int base = 0; base < total; base += 128 * kBatch) {
          float4 v[kBatch];
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int c = base + u * 128 + pt;
            const int rq = c % (t.tn / 4), kk = c / (t.tn / 4);
            const int nr = n0 + rq * 4, kr = k0 + kk;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c < total && nr < t.nr && kr < kend) {
              const int tt = nr >= d.N;
              const int n = nr - tt * d.N;
              int sk = 0, k = kr;
              if (!t.quad) { sk = kr >= K; k = kr - sk * K; }
              int64_t off = (int64_t)n * d.b_n + koff(k, d.K2, d.b_k1, d.b_k2);
              float sign = 1.f;
              if (t.quad) { off += tt ? d.plane_b : 0; }
              else if (sk != tt) {
                off += d.plane_b;
                sign = (d.conj_b ? -1.f : 1.f) * (sk == 0 ? 1.f : -1.f);
              }
              v[u] = __ldg(reinterpret_cast<const float4*>(B + off));
              v[u].x *= sign; v[u].y *= sign; v[u].z *= sign; v[u].w *= sign;
            }
          }
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int c = base + u * 128 + pt;
            if (c >= total) continue;
            const int row = (c % (t.tn / 4)) * 4, kk = c / (t.tn / 4);
            store_elem(tb, row, kk, v[u].x, t.bf16);
            store_elem(tb, row + 1, kk, v[u].y, t.bf16);
            store_elem(tb, row + 2, kk, v[u].z, t.bf16);
            store_elem(tb, row + 3, kk, v[u].w, t.bf16);
            if (t.x3) {
              const float4 l = lo_part4(v[u], t.bf16);
              store_elem(tbl, row, kk, l.x, t.bf16);
              store_elem(tbl, row + 1, kk, l.y, t.bf16);
              store_elem(tbl, row + 2, kk, l.z, t.bf16);
              store_elem(tbl, row + 3, kk, l.w, t.bf16);
            }
          }
        }
      } else {
        for (int i = pt; i < t.tn * kelems; i += 128) {
          int row, kk;
          if (b_nfast) { row = i % t.tn; kk = i / t.tn; }
          else { kk = i % kelems; row = i / kelems; }
          const int nr = n0 + row, kr = k0 + kk;
          const float v = (nr < t.nr && kr < kend) ? load_b(d, t, B, nr, kr) : 0.f;
          store_elem(tb, row, kk, v, t.bf16);
          if (t.x3) store_elem(tbl, row, kk, lo_part(v, t.bf16), t.bf16);
        }
      }
      if (!(a_async && b_async)) fence_proxy_async();  // generic-proxy stores of this stage
      if (a_async || b_async) cp_async_arrive(&full[s]);
      else mbar_arrive(&full[s]);
    }
  } else if (warp == 0) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t idesc = make_idesc(t.bf16 ? 1 : 2, kTM, t.tn);
      for (int kt = 0; kt < ntiles; ++kt) {
        const int s = kt % kStages;
        const bool ok = mbar_wait(&full[s], (kt / kStages) & 1, t.err);
        if (!ok) *abort_flag = 1;
        if (!*abort_flag) {
          // the stage was written through the generic proxy (cp.async, st.shared);
          // order those writes before the tensor core's async-proxy reads
          fence_proxy_async();
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + s * TcSmem::kA);
          const uint32_t b0 = smem_u32(sB + s * TcSmem::kB);
          const uint32_t al = smem_u32(sAl + s * TcSmem::kA);
          const uint32_t bl = smem_u32(sBl + s * TcSmem::kB);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {  // 4 x 32 bytes of K per 128-byte row
            mma_issue(t.bf16, tmem, sw128_desc(a0 + ks * 32), sw128_desc(b0 + ks * 32), idesc,
                      (kt > 0 || ks > 0) ? 1u : 0u);
            if (t.x3) {
              mma_issue(t.bf16, tmem, sw128_desc(a0 + ks * 32), sw128_desc(bl + ks * 32), idesc, 1u);
              mma_issue(t.bf16, tmem, sw128_desc(al + ks * 32), sw128_desc(b0 + ks * 32), idesc, 1u);
            }
          }
        }
        mma_commit(&empty[s]);
      }
      mma_commit(accum);
    }
    __syncwarp();
  }

  // -------------------------------------------------------------- epilogue
  if (warp < 4) {
    const bool ok = mbar_wait(accum, 0, t.err);
    tc_fence_after();
    __syncwarp();
    const int row = warp * 32 + lane;  // accumulator row = TMEM lane
    const int mr = m0 + row;
    float* C = d.C[outer] + inner * d.c_in;
    if (!t.quad && t.splits > 1) {
      // split-K partial [split][outer][inner][re|im][M][N] (an empty split writes zeros)
      float* q = t.part + ((((int64_t)split * d.n_outer + outer) * d.n_inner + inner) * 2) *
                              (int64_t)d.M * d.N;
      for (int c0 = 0; c0 < t.tn; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
        if (mr >= t.mr) continue;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int nr = n0 + c0 + j;
          if (nr >= t.nr) break;
          const int tt = nr >= d.N;
          const int n = nr - tt * d.N;
          q[(int64_t)tt * d.M * d.N + (int64_t)mr * d.N + n] = (ok && ntiles > 0) ? v[j] : 0.f;
        }
      }
    } else if (!t.quad) {
      for (int c0 = 0; c0 < t.tn; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
        if (!ok || ntiles == 0 || mr >= t.mr) continue;
        const int nb = n0 + c0;
        const int tt0 = nb >= d.N;
        if (d.c_n == 1 && !d.accumulate && nb + 32 <= t.nr && (nb - tt0 * d.N) + 32 <= d.N) {
          float* p = C + ROW_C(d, mr) + (nb - tt0 * d.N) + (tt0 ? d.plane_c : 0);
          if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
              *reinterpret_cast<float4*>(p + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            continue;
          }
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int nr = n0 + c0 + j;
          if (nr >= t.nr) break;
          const int tt = nr >= d.N;
          const int n = nr - tt * d.N;
          float* p = C + ROW_C(d, mr) + (int64_t)n * d.c_n + (tt ? d.plane_c : 0);
          if (d.accumulate) *p += v[j]; else *p = v[j];
        }
      }
    } else {
      // stage P in shared memory (the pipeline buffers are free now), then combine
      float* P = reinterpret_cast<float*>(smem);  // [128][tn + 1]
      const int ld = t.tn + 1;
      for (int c0 = 0; c0 < t.tn; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < t.tn) P[row * ld + c0 + j] = v[j];
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      const float sa = d.conj_a ? -1.f : 1.f, sb = d.conj_b ? -1.f : 1.f;
      const int M = d.M, N = d.N;
      const bool valid = ok && ntiles > 0;  // an empty K split contributes zeros
      for (int idx = tid; idx < M * N; idx += 128) {
        const int m = idx / N, n = idx - (idx / N) * N;
        float cr = 0.f, ci = 0.f;
        if (valid) {
          const float prr = P[m * ld + n], pii = P[(M + m) * ld + N + n];
          const float pri = P[m * ld + N + n], pir = P[(M + m) * ld + n];
          cr = prr - sa * sb * pii;
          ci = sb * pri + sa * pir;
        }
        if (t.splits > 1) {
          float* q = t.part + ((((int64_t)split * d.n_outer + outer) * d.n_inner + inner) * 2) *
                                  (int64_t)M * N;
          q[(int64_t)m * N + n] = cr;
          q[(int64_t)M * N + (int64_t)m * N + n] = ci;
        } else if (valid) {
          float* p = C + ROW_C(d, m) + (int64_t)n * d.c_n;
          if (d.accumulate) { p[0] += cr; p[d.plane_c] += ci; }
          else { p[0] = cr; p[d.plane_c] = ci; }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// Sum the K-split partials in a fixed order and store C.
__global__ void tc_reduce_kernel(GemmDesc d, const float* part, int splits) {
  const int z = blockIdx.y;
  const int outer = z / d.n_inner, inner = z - outer * d.n_inner;
  if (outer_frozen(d, outer)) return;
  const int M = d.M, N = d.N;
  float* C = d.C[outer] + inner * d.c_in;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < M * N; idx += gridDim.x * blockDim.x) {
    const int m = idx / N, n = idx - m * N;
    // partials summed in FP64 in split order, rounded once
    double cr = 0.0, ci = 0.0;
    for (int s = 0; s < splits; ++s) {
      const float* q =
          part + ((((int64_t)s * d.n_outer + outer) * d.n_inner + inner) * 2) * (int64_t)M * N;
      cr += (double)q[idx];
      ci += (double)q[(int64_t)M * N + idx];
    }
    float* p = C + ROW_C(d, m) + (int64_t)n * d.c_n;
    if (d.accumulate) { p[0] = (float)((double)p[0] + cr); p[d.plane_c] = (float)((double)p[d.plane_c] + ci); }
    else { p[0] = (float)cr; p[d.plane_c] = (float)ci; }
  }
}

}  // namespace

size_t tc_smem_bytes(int x3) { return TcSmem::bytes(x3) + 1024; }

// Sum split-K partials [split][outer][inner][re|im][M][N] into C in a fixed order.
cudaError_t launch_tc_reduce(const GemmDesc& d, const float* part, int splits, cudaStream_t st) {
  dim3 rg((d.M * d.N + 255) / 256, d.n_outer * d.n_inner);
  tc_reduce_kernel<<<rg, 256, 0, st>>>(d, part, splits);
  return cudaGetLastError();
}

// Plan a tensor-core launch for d: quad form when the contraction is long and
// M, N small (2M <= 128), else realified-B form.
bool tc_plan(const GemmDesc& d, int* quad, int* splits, size_t* part_floats, int force_splits) {
  const int64_t K = (int64_t)d.K1 * d.K2;
  *quad = (2 * d.M <= kTM && 2 * d.N <= kTN && !d.b_pre) ? 1 : 0;
  *splits = 1;
  *part_floats = 0;
  const int kel = (d.prec == TN_BF16 || d.prec == TN_BF16X3) ? 64 : 32;
  const int64_t batch = (int64_t)d.n_outer * d.n_inner;
  if (*quad) {
    const int64_t tiles = (K + kel - 1) / kel;
    int s = 1;
    while (batch * s < 2 * 152 && s * 2 <= tiles / 4 && s < 64) s *= 2;
    *splits = s;
  } else {
    // realified-B form: split K when the output tiles alone leave most of the
    // GPU idle (a few sites with a long contraction: the closes of a small
    // cell at large chi)
    const int64_t nr = 2 * (int64_t)d.N;
    const int64_t tn = nr >= kTN ? kTN : ((nr + 15) / 16) * 16;
    const int64_t ctas = batch * ((d.M + kTM - 1) / kTM) * ((nr + tn - 1) / tn);
    const int64_t ktiles = (2 * K + kel - 1) / kel;
    int s = 1;
    if (ctas < 152)
      while (ctas * s < 2 * 152 && s * 2 <= ktiles / 4 && s < 64) s *= 2;
    *splits = s;
  }
  if (force_splits > 0) {
    // the autotuner's count, at most one K tile per split
    const int64_t kt = *quad ? (K + kel - 1) / kel : (2 * K + kel - 1) / kel;
    *splits = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)force_splits, 64, kt}));
  }
  if (*splits > 1) *part_floats = (size_t)(*splits) * batch * 2 * d.M * d.N;
  return true;
}

// Kernel attributes, set once before any launch (and before any stream capture).
cudaError_t tc_prepare() {
  static std::once_flag once;
  static cudaError_t result = cudaSuccess;
  std::call_once(once, [] {
    result = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc_smem_bytes(1));
    // two CTAs per SM: ask for the largest shared-memory carveout
    if (result == cudaSuccess)
      result = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    100);
  });
  return result;
}

cudaError_t launch_cgemm_tc(const GemmDesc& d, float* part, int* err, cudaStream_t st,
                            int* n_kernels, int force_splits, size_t part_cap) {
  if (n_kernels) *n_kernels = 0;
  if (d.M <= 0 || d.N <= 0 || d.n_outer <= 0 || d.n_inner <= 0) return cudaSuccess;
  int quad, splits;
  size_t pf;
  if (!tc_plan(d, &quad, &splits, &pf, force_splits)) return cudaErrorInvalidValue;
  if (splits > 1 && (!part || pf > part_cap)) return cudaErrorInvalidValue;
  TcArgs t;
  t.quad = quad;
  t.bf16 = (d.prec == TN_BF16 || d.prec == TN_BF16X3) ? 1 : 0;
  t.x3 = (d.prec == TN_TF32X3 || d.prec == TN_BF16X3) ? 1 : 0;
  const int64_t K = (int64_t)d.K1 * d.K2;
  if (quad) { t.mr = 2 * d.M; t.nr = 2 * d.N; t.kr = (int)K; }
  else { t.mr = d.M; t.nr = 2 * d.N; t.kr = (int)(2 * K); }
  t.tn = t.nr >= kTN ? kTN : ((t.nr + 15) / 16) * 16;
  const int kel = t.bf16 ? 64 : 32;
  t.splits = splits;
  const int64_t tiles = (t.kr + kel - 1) / kel;
  t.k_per_split = (int)(((tiles + splits - 1) / splits) * kel);
  t.part = part;
  t.err = err;
  {
    cudaError_t e = tc_prepare();
    if (e != cudaSuccess) return e;
  }
  dim3 grid((t.nr + t.tn - 1) / t.tn, (t.mr + kTM - 1) / kTM, d.n_outer * d.n_inner * splits);
  tc_gemm_kernel<<<grid, kThreads, tc_smem_bytes(t.x3), st>>>(d, t);
  if (n_kernels) *n_kernels = splits > 1 ? 2 : 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  dim3 rg((d.M * d.N + 255) / 256, d.n_outer * d.n_inner);
  tc_reduce_kernel<<<rg, 256, 0, st>>>(d, part, splits);
  return cudaGetLastError();
}

}  // namespace tnbp
