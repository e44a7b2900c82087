// S3+S4 R_II contraction on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// For one (height z, scattering-angle class c, chunk of <= 32 output
// directions) the CTA computes the real product
//     eps_bar[n][(o,i)] += sum_{ti, k} A[ti][n][k] * B[ti][k][(o,i)],   k in [0, 2N)
// where A[ti] is the stored tile (Re | Im halves of the tile against the spline
// basis, Eq. RQIIKKp / Eq. G) and
//     B[ti][k][(o,i)] = sum_{o' in class, j} Ycomp_{ti,ij}(o,o') I~_j(o', m)
// with Ycomp = Re Y for k = m < N and -Im Y for k = N + m (so that the sum is
// Re(T Z) over the complex tile T and Z = Y I~).  The MMA computes the
// transpose, D[(o,i)][n] = sum_k B^T[(o,i)][k] A^T[k][n]: M = 128 Stokes
// columns, N = all tile rows n (<= 256, padded to 16), so one MMA per K
// slice covers a whole tile step without padding n to a second M block.
//
// Roles (320 threads): warp 0 streams the tile into a 5-stage ring with one
// bulk asynchronous copy per K step (the FP32 tiles are stored pre-swizzled, K
// step by K step, so a step is one contiguous N x 64-byte block), stages the
// step's I~ of every incident direction of the CTA beside it (one or two bulk
// copies per direction, issued by its 32 lanes, completing on the same stage
// barrier) and owns the TMEM allocation; warp 1 issues tcgen05.mma; warps 2-9 build B in shared memory
// from Y (staged per tile, prefetched into registers a tile ahead) and the
// staged I~, split both operands into TF32 hi/lo parts
// (3 products: hi*hi + hi*lo + lo*hi, FP32-level accuracy) in a 2-buffer ring
// of their own, and run the epilogue from TMEM.  The tile ring is deeper than
// the builder ring so that enough tile bytes are in flight per SM to cover
// HBM latency at full bandwidth.
// Accumulator: 128 TMEM lanes x NM columns.  Every mbarrier wait is bounded; on
// expiry the CTA records an error flag, drains what it issued and returns.
#include <algorithm>
#include <cstdio>
#include <vector>
#include <cuda_bf16.h>
#include "prd_internal.h"
#include "device_common.cuh"

namespace prd {

namespace tc {

constexpr int kStagesMax = 5;                 // tile ring depth: 2..5, the most that fit beside the rest
constexpr int kCBufsMax = 4;                  // builder ring (A_lo, B_hi, B_lo): 2 buffers, 4 for split tiles
constexpr int kKC = 16;                       // fp32 per stage along K (64-byte rows)
constexpr int kMaxE = 32;                     // output directions per CTA
constexpr int kNCPMax = 4 * kMaxE;            // MMA N (Stokes columns)
constexpr int kBBytes = kNCPMax * kKC * 4;
__host__ __device__ constexpr int n_cbufs(bool split) { return split ? 4 : 2; }
// Builder warps: the B build and the TF32 splits are chains of dependent
// shared-memory loads and FMAs, so the builders are latency-bound; more warps
// hide more of that latency (16 warps, one B item each, fit 576 threads x 112
// registers).
constexpr int kGenWarps = 16;
constexpr int kGen = 32 * kGenWarps;          // builder threads (warps 2 .. 2 + kGenWarps - 1)
constexpr int kThreads = 64 + kGen;
constexpr int kItems = 16 / kGenWarps;        // B items per builder warp (16 items of 32 rows x 4 k)
constexpr int kYPairsC = 64;
constexpr int kYR = (kYPairsC * 8 + kGen - 1) / kGen;   // Y prefetch float4 per builder thread
constexpr int kAR = (1024 + kGen - 1) / kGen;           // A_lo float4 per builder thread (N <= 256)
constexpr int kYPairs = kYPairsC;             // pairs whose Y is staged in shared memory
constexpr int kYBytes = kYPairs * 32 * 4;     // one tile's Y (two buffers)
constexpr int kISlots = 32;                   // incident directions whose I~ is resident per CTA
constexpr int kAuxBytes = 1024;               // work-item tables, barriers, TMEM slot, abort flag
constexpr int kSmemMax = 227 * 1024;          // shared memory per CTA
static_assert(kNCPMax == 128 && (kGenWarps == 8 || kGenWarps == 16), "B items: 16 (32-row group, 4-k chunk) over the builder warps");
// Shared memory of one CTA for N tile rows with `st` tile stages: the tile ring
// (NM x 64 bytes per K step), the builder ring (A_lo of NM rows unless the
// tiles come split, B_hi, B_lo), two Y buffers, the resident I~ of kISlots
// incident directions (stride N + 1 float4, odd modulo 8 so that different
// slots fall in different bank groups) and the auxiliary tables, plus 1 KB to
// align the base.
// (split tiles: no A_lo, and the B planes are bf16, 4 KB each)
__host__ __device__ constexpr int cbuf_bytes(int N, bool split) {
  return split ? kBBytes : ((N + 15) / 16 * 16) * 64 + 2 * kBBytes;
}
__host__ __device__ constexpr int smem_bytes(int N, int st, bool split) {
  return st * ((N + 15) / 16 * 16) * 64 + n_cbufs(split) * cbuf_bytes(N, split) + 2 * kYBytes +
         kISlots * ((N + 15) / 16 * 16 + 1) * 16 +
         kAuxBytes + 1024;
}
constexpr long long kSpin = 1ll << 24;        // bounded waits (default limit of the pipeline waits; drains)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\tselp.b32 %0, 1, 0, P;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded pipeline wait of at most `limit` polls; returns false (and raises the
// CTA abort flag) on expiry or when another role has aborted
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, long long limit) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_try(b, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// bulk asynchronous copy global -> shared (16-byte aligned ends, size a multiple
// of 16) with an L2 eviction-priority policy
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
      ::"r"(smem_u32(dst)), "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
// the tiles are streamed once per apply: first out of L2, so that I~ and Y stay resident
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 B apart
__device__ __forceinline__ uint64_t sdesc(const void* p) {
  const uint64_t addr = (smem_u32(p) & 0x3FFFF) >> 4;
  const uint64_t lbo = 1;            // unused for swizzled K-major
  const uint64_t sbo = 512 >> 4;
  return addr | (lbo << 16) | (sbo << 32) | (1ull << 46) | (4ull << 61);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
      ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// BF16 operands (kind::f16), FP32 accumulation, K = 16 per instruction
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// shared-memory matrix descriptor: K-major, 32-byte swizzle (rows of 16 bf16),
// 8-row groups 256 B apart
__device__ __forceinline__ uint64_t sdesc32(const void* p) {
  const uint64_t addr = (smem_u32(p) & 0x3FFFF) >> 4;
  const uint64_t lbo = 1;            // unused for swizzled K-major
  const uint64_t sbo = 256 >> 4;
  return addr | (lbo << 16) | (sbo << 32) | (1ull << 46) | (6ull << 61);
}
// byte offset of the 4 bf16 of k-group g (k = 4g .. 4g + 3, g < 4) of `row` in a
// K-major 32-byte-swizzled operand: the 16-byte half (g >> 1) is exchanged with
// the other in rows whose bit 2 is set
__device__ __forceinline__ uint32_t swz32(int row, int g) {
  return (uint32_t)row * 32u + (uint32_t)(((g >> 1) ^ ((row >> 2) & 1)) * 16) + (uint32_t)(g & 1) * 8u;
}
// v split into bf16 hi = rn(v) and lo = rn(v - hi): |v - hi - lo| <= 2^-18 |v|;
// the three products hi*hi + hi*lo + lo*hi then leave <= 3 * 2^-18 |a b|
__device__ __forceinline__ void bf16_split4(float4 v, uint2& hi, uint2& lo) {
  const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y), h1 = __floats2bfloat162_rn(v.z, v.w);
  const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
  const __nv_bfloat162 l0 = __floats2bfloat162_rn(v.x - f0.x, v.y - f0.y);
  const __nv_bfloat162 l1 = __floats2bfloat162_rn(v.z - f1.x, v.w - f1.y);
  hi.x = *reinterpret_cast<const uint32_t*>(&h0);
  hi.y = *reinterpret_cast<const uint32_t*>(&h1);
  lo.x = *reinterpret_cast<const uint32_t*>(&l0);
  lo.y = *reinterpret_cast<const uint32_t*>(&l1);
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// v rounded to TF32 (nearest, ties away from zero: half a unit of the 13
// dropped bits is added to the magnitude bits before they are cleared).  The
// tensor pipe drops the low 13 bits of a raw FP32 operand.  B is split as
// hi = rna(v), lo = rna(v - hi): v - hi is exact in FP32 and |v - hi| <= 2^-11 |v|,
// so |v - hi - lo| <= 2^-22 |v|.  A (the stored tile, read raw) has the
// truncated hi = trunc(a) and lo = rna(a - trunc(a)) with |a - trunc(a)| < 2^-10 |a|,
// so |a - hi - lo| <= 2^-21 |a|; the dropped lo*lo term is below 2^-21 |a b|.
__device__ __forceinline__ float tf32_hi(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ float tf32_trunc(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

// byte offset of element (row, k) in a K-major 64-byte-swizzled operand (k < 16)
__device__ __forceinline__ uint32_t swz64(int row, int k) {
  const uint32_t chunk = (uint32_t)(k >> 2) ^ (uint32_t)((row >> 1) & 3);
  return (uint32_t)((row >> 3) * 512 + (row & 7) * 64) + chunk * 16 + (uint32_t)(k & 3) * 4;
}

struct Params {
  const float* tiles;   // [z][class][tile] pre-swizzled K steps of [N][16]
  const float* Y;       // [z][pair][ntile][16][2]
  const float* Ic;      // [z][o][N][4]
  const int2* work;     // [item] (class, first output entry of the chunk)
  const int* cls;
  float* eb;            // [z][o][N][4]
  int* err;
  int ncls, ntile, nO, N, npairs, ld;
  int nst;              // tile stages (2..kStagesMax)
  long long spin;       // poll limit of the pipeline waits (the drains keep kSpin)
};

// barrier over the builder warps only (named barrier 1)
__device__ __forceinline__ void gen_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kGen) : "memory"); }
// same barrier, returning whether v holds on every builder thread (keeps the
// builders' loop exits uniform, so none waits at the barrier for one that left)
__device__ __forceinline__ bool gen_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\tbar.red.and.pred q, 1, %2, p;\n\tselp.b32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kGen)
      : "memory");
  return r != 0;
}

// kBF16: the split-BF16 products (BF16x3) instead of 3xTF32, operands K-major
// with 32-byte rows (16 bf16 of K).  kSplit (with kBF16): the tiles are stored
// split (tile_off_split), so the producer's two bulk copies per step land the
// hi and lo planes in the operand layout and the builders never touch the
// tile; without it the builders split the FP32 tile step into the planes.
// kHi (with kSplit): the tiles hold the hi plane alone (BF16x2 contexts, half
// the bytes) and each step is the two products hi*hi + lo(B)*hi.
template <bool kBF16, bool kSplit, bool kHi>
__global__ void __launch_bounds__(kThreads, 1) r2_tc_kernel(Params p) {
  static_assert(kBF16 || !kSplit, "split tiles are bf16 planes");
  static_assert(kSplit || !kHi, "hi-only tiles are split tiles");
  extern __shared__ __align__(1024) unsigned char smraw[];
  // 1024-byte aligned base, derived by offset so that the compiler keeps the
  // shared address space on every pointer below (plain LDS/STS, no generic access)
  unsigned char* sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
  const int N = p.N;
  const int NM = (N + 15) / 16 * 16;             // MMA N: the tile rows n (<= 256)
  const int SA = NM * kKC * 4;                   // one K step of the tile (multiple of 1024 bytes)
  const int nst = p.nst;
  const int NP = p.ld >> 1;                      // padded half width (N rounded up to 16)
  const int IS = NP + 1;                         // float4 stride of a resident I~ slot (zero for k >= N)
  unsigned char* cbuf = sm + nst * SA;                             // [buffer] A_lo, B_hi, B_lo
  const int CB = cbuf_bytes(N, kSplit);
  constexpr int NCB = n_cbufs(kSplit);                             // builder ring depth
  constexpr int BPL = kSplit ? kBBytes / 2 : kBBytes;              // bytes of one B plane
  float* Ys = (float*)(cbuf + NCB * CB);                           // [buffer][pair][16][2]
  float4* Ir = (float4*)((unsigned char*)Ys + 2 * kYBytes);         // [slot][k < N], resident
  int* eptr = (int*)((unsigned char*)Ir + (size_t)kISlots * IS * 16);   // local pair range of each output
  int* fast_p = eptr + kMaxE + 1;                                  // fast-path flag, staged slots
  int* pslot = fast_p + 2;                                         // slot of each local pair
  int* slot_dir = pslot + kYPairs;                                 // direction held in each slot
  uint64_t* full = (uint64_t*)(((uintptr_t)(slot_dir + kISlots) + 7) & ~(uintptr_t)7);
  uint64_t* empty = full + kStagesMax;
  uint64_t* ready = empty + kStagesMax;
  uint64_t* cfree = ready + kCBufsMax;
  uint64_t* done = cfree + kCBufsMax;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int2 wk = p.work[blockIdx.x];
  const int c = wk.x, e0 = wk.y, iz = blockIdx.y;
  const int* cout_ptr = p.cls;
  const int* cout_dir = p.cls + p.ncls + 1;
  const int ne_tot = cout_ptr[p.ncls];
  const int* pair_ptr = cout_dir + ne_tot;
  const int* pair_in = pair_ptr + ne_tot + 1;
  const int E = min(kMaxE, cout_ptr[c + 1] - e0);
  const int NCP = ((4 * E + 15) / 16) * 16;      // MMA N (multiple of 16, <= 128)
  const int KCH = p.ld / kKC;                    // K steps per tile: KH of the Re half, then KH of the Im half
  const int KH = KCH >> 1;
  const int iters = p.ntile * KCH;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gt = threadIdx.x - 64;               // builder thread index (warps 2..)
  const uint32_t tm_cols = 256u;                 // D: 128 lanes x NM (<= 256) columns
  const int pp0 = pair_ptr[e0], npl = pair_ptr[e0 + E] - pp0;
  const bool y_in_smem = npl <= kYPairs;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);        // armed by the producer with the bytes of the tile copy
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NCB; ++b) {
      mbar_init(&ready[b], kGen);
      mbar_init(&cfree[b], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (gt >= 0 && gt <= E) eptr[gt] = pair_ptr[e0 + gt] - pp0;
  // incident directions of this CTA's pairs -> I~ slots (first kISlots distinct); the
  // fast path needs every pair's Y and I~ staged and at most two pairs per output
  if (gt == 0) {
    int ns = 0;
    bool all = y_in_smem;
    for (int el = 0; el < E; ++el) all = all && pair_ptr[e0 + el + 1] - pair_ptr[e0 + el] <= 2;
    for (int pl = 0; pl < npl && pl < kYPairs; ++pl) {
      const int op = pair_in[pp0 + pl];
      int sidx = -1;
      for (int s2 = 0; s2 < ns; ++s2)
        if (slot_dir[s2] == op) { sidx = s2; break; }
      if (sidx < 0 && ns < kISlots) { slot_dir[ns] = op; sidx = ns++; }
      pslot[pl] = sidx;
      all = all && sidx >= 0;
    }
    fast_p[0] = all ? 1 : 0;
    fast_p[1] = ns;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tm_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const bool fast = fast_p[0] != 0;
  const int ns = fast_p[1];
  const long long slab0 = ((long long)iz * p.ncls + c) * p.ntile;
  const float* Icz = p.Ic + (size_t)iz * p.nO * N * 4;

  if (warp == 0) {
    // ---------------- producer: lane 0 waits for a free stage, arms its barrier with the
    // bytes of the step and copies the tile K step (one bulk copy), up to nst steps
    // ahead of the MMAs.  I~ is resident (staged once by the builders).
    if (lane == 0) {
      int it = 0;
      const uint64_t pol_t = policy_evict_first();
      // bytes of one K step of the stored tile: N rows x 64 (FP32, or the two bf16
      // planes), N x 32 (hi plane alone)
      const uint32_t abytes = (uint32_t)N * kKC * (kHi ? 2 : 4);
      // stage s = it % nst with phase parity ps = (it / nst) & 1, tile ti = it / KCH and
      // its K step kc, all advanced incrementally (no divisions per step)
      int s = 0, ps = 0, ti = 0, kc = 0;
      for (; it < iters; ++it, s = (s + 1 == nst) ? (ps ^= 1, 0) : s + 1, kc = (kc + 1 == KCH) ? (++ti, 0) : kc + 1) {
        if (it >= nst && !mbar_wait(&empty[s], ps ^ 1, abort_flag, p.spin)) break;
        // rows n >= N of the stage keep stale data: they only reach output rows
        // that the epilogue never reads
        const unsigned char* src = reinterpret_cast<const unsigned char*>(p.tiles) +
                                   ((size_t)(slab0 + ti) * N * p.ld + (size_t)kc * N * kKC) * (kHi ? 2 : 4);
        mbar_expect_tx(&full[s], abytes);
        if constexpr (kHi) {
          bulk_load(sm + s * SA, src, abytes, &full[s], pol_t);          // hi plane at the stage
        } else if constexpr (kSplit) {
          // hi plane (N x 32 bytes) at the stage, lo plane at its second half
          bulk_load(sm + s * SA, src, abytes / 2, &full[s], pol_t);
          bulk_load(sm + s * SA + SA / 2, src + abytes / 2, abytes / 2, &full[s], pol_t);
        } else {
          bulk_load(sm + s * SA, src, abytes, &full[s], pol_t);
        }
      }
      if (*abort_flag) {
        // drain copies that were issued and may not have been consumed
        for (int j = max(0, it - nst); j < it; ++j) {
          const int s = j % nst;
          for (long long i = 0; i < kSpin && !mbar_try(&full[s], (j / nst) & 1); ++i) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      // D[(o,i)][n] (M = 128 Stokes columns of the chunk, N = NM tile rows): the built
      // operand is A, the streamed tile is B, so one MMA covers every row n
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NM >> 3) << 17) | ((128u >> 4) << 24);
      int issued = 0;
      int s = 0, ps = 0;                         // it % nst and (it / nst) & 1
      for (int it = 0; it < iters; ++it, s = (s + 1 == nst) ? (ps ^= 1, 0) : s + 1) {
        const int cb = it & (NCB - 1);
        if (!mbar_wait(&ready[cb], (it / NCB) & 1, abort_flag, p.spin)) break;
        // split tiles: the builders do not wait for the tile step, the MMAs do
        if (kSplit && !mbar_wait(&full[s], ps, abort_flag, p.spin)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned char* A = sm + s * SA;
        unsigned char* Alo = cbuf + cb * CB;
        unsigned char* Bhi = Alo + (kSplit ? 0 : SA);
        unsigned char* Blo = Bhi + BPL;
        if constexpr (kBF16) {
          // A_hi and A_lo planes (NM x 32 bytes each): the stage itself for split
          // tiles, else the A_lo buffer the builders filled
          const uint32_t idesc16 =
              (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NM >> 3) << 17) | ((128u >> 4) << 24);
          unsigned char* Ah = kSplit ? A : Alo;
          unsigned char* Al = Ah + SA / 2;
          mma_bf16(tmem, sdesc32(Bhi), sdesc32(Ah), idesc16, it > 0 ? 1u : 0u);
          mma_bf16(tmem, sdesc32(Blo), sdesc32(Ah), idesc16, 1u);
          if constexpr (!kHi) mma_bf16(tmem, sdesc32(Bhi), sdesc32(Al), idesc16, 1u);
        } else {
          for (int ks = 0; ks < 2; ++ks) {
            const int o = ks * 32;                 // 8 fp32 of K per MMA
            const uint32_t acc = (it > 0 || ks > 0) ? 1u : 0u;
            mma_tf32(tmem, sdesc(Bhi + o), sdesc(A + o), idesc, acc);
            mma_tf32(tmem, sdesc(Blo + o), sdesc(A + o), idesc, 1u);
            mma_tf32(tmem, sdesc(Bhi + o), sdesc(Alo + o), idesc, 1u);
          }
        }
        mma_commit(&empty[s]);
        mma_commit(&cfree[cb]);
        issued = it + 1;
      }
      if (issued > 0) {
        mma_commit(done);
        // on abort, let the MMAs already issued finish before TMEM is released
        if (*abort_flag)
          for (long long i = 0; i < kSpin && !mbar_try(done, 0); ++i) {
          }
      } else {
        *abort_flag = 1;
      }
    }
  } else {
    // ---------------- B builders / A splitters, then epilogue
    const int bw = warp - 2;                       // builder warp
    // B items: (32-row group rg, 4-k chunk kq), item = bw + 8 r over the 4 nrg items
    // of the chunk, so every builder warp has work whatever the chunk's width; a
    // lane takes row rg*32 + lane (output el = row / 4, Stokes i = row % 4), and
    // the swizzle spreads each 8 lanes' stores over all banks
    const int nrg = (NCP + 31) / 32;
    int it_row[kItems], it_kq[kItems], it_pa[kItems], it_pb[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int item = bw + kGenWarps * r;
      const bool vi = item < nrg * 4;
      const int rg = vi ? item % nrg : 0;
      it_row[r] = vi ? rg * 32 + lane : NCP;      // NCP: no item
      it_kq[r] = vi ? item / nrg : 0;
      const int el = it_row[r] >> 2;
      const bool v = it_row[r] < NCP && el < E;
      it_pa[r] = v ? eptr[el] : 0;
      it_pb[r] = v ? eptr[el + 1] : 0;
    }
    const size_t ybase = (size_t)iz * p.npairs + pp0;
    float4 ypre[kYR];
    auto load_y = [&](int ti) {
#pragma unroll
      for (int r = 0; r < kYR; ++r) {
        const int q = gt + r * kGen;
        if (y_in_smem && q < npl * 8)
          ypre[r] = *((const float4*)(p.Y + ((ybase + (q >> 3)) * p.ntile + ti) * 32) + (q & 7));
      }
    };
    // fast path: each lane keeps, per item and pair, the four coefficients of the
    // current half (Re Y_ij for the Re half, -Im Y_ij for the Im half) and the I~
    // slot offset in registers.  I~ does not depend on the tile: column k of either
    // half reads I~(k).  So the I~ of the CTA's staged incident directions is loaded
    // into shared memory once, here (zero for N <= k < NP, so the padded columns
    // need no test), while the producer already streams the first tile steps.
    float4 ycf[kItems][2];
    int soff[kItems][2];
    load_y(0);
    {
      const float4* Icz4 = reinterpret_cast<const float4*>(Icz);
      for (int idx = gt; idx < ns * NP; idx += kGen) {
        const int sl = idx / NP, k = idx - sl * NP;
        Ir[sl * IS + k] = k < N ? Icz4[(size_t)slot_dir[sl] * N + k] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      gen_sync();
    }
    // the coefficients of item r's pairs for the Re (im = false) or Im half of the tile in Ysb
    auto load_cf = [&](const float* Ysb, bool im) {
#pragma unroll
      for (int r = 0; r < kItems; ++r) {
        const int npr = it_pb[r] - it_pa[r], i = it_row[r] & 3;
#pragma unroll
        for (int pp = 0; pp < 2; ++pp)
          if (pp < npr) {
            const float4* y4 = reinterpret_cast<const float4*>(Ysb) + (it_pa[r] + pp) * 8 + i * 2;
            const float4 ya = y4[0], yb = y4[1];
            ycf[r][pp] = im ? make_float4(-ya.y, -ya.w, -yb.y, -yb.w) : make_float4(ya.x, ya.z, yb.x, yb.z);
          }
      }
    };
    bool aborted = false;
    int s = 0, ps = 0, ti = 0, kc = 0;           // it % nst, (it / nst) & 1, it / KCH, it % KCH
    for (int it = 0; it < iters;
         ++it, s = (s + 1 == nst) ? (ps ^= 1, 0) : s + 1, kc = (kc + 1 == KCH) ? (++ti, 0) : kc + 1) {
      const int cb = it & (NCB - 1);
      bool got = !aborted && (kSplit || mbar_wait(&full[s], ps, abort_flag, p.spin));
      if (got && it >= NCB) got = mbar_wait(&cfree[cb], ((it / NCB) - 1) & 1, abort_flag, p.spin);
      float* Ysb = Ys + (ti & 1) * (kYPairs * 32);
      if (kc == 0) {
        // a new tile: stage its Y, then all builders agree to go on (every builder
        // reaches this barrier, aborted or not, so none waits for one that left)
#pragma unroll
        for (int r = 0; r < kYR; ++r) {
          const int q = gt + r * kGen;
          if (y_in_smem && q < npl * 8) ((float4*)Ysb)[q] = ypre[r];
        }
        got = gen_all(got);
        if (got && fast) {
          load_cf(Ysb, false);
#pragma unroll
          for (int r = 0; r < kItems; ++r) {
            const int npr = it_pb[r] - it_pa[r];
#pragma unroll
            for (int pp = 0; pp < 2; ++pp)
              if (pp < npr) soff[r][pp] = pslot[it_pa[r] + pp] * IS;
          }
        }
        if (ti + 1 < p.ntile) load_y(ti + 1);
      } else if (kc == KH && got && fast) {
        load_cf(Ysb, true);                        // the Im half of the tile begins
      }
      if (!got) {
        aborted = true;
        continue;
      }
      unsigned char* A = sm + s * SA;
      unsigned char* Alo = cbuf + cb * CB;
      unsigned char* Bhi = Alo + (kSplit ? 0 : SA);
      unsigned char* Blo = Bhi + BPL;
      if constexpr (!kSplit) {
        const float4* a4 = (const float4*)A;
        float4* l4 = (float4*)Alo;
        const int nq4 = N * (kKC / 4);             // <= kAR kGen
        float4 v[kAR];
#pragma unroll
        for (int r = 0; r < kAR; ++r)
          if (gt + r * kGen < nq4) v[r] = a4[gt + r * kGen];
#pragma unroll
        for (int r = 0; r < kAR; ++r)
          if (gt + r * kGen < nq4) {
            if constexpr (kBF16) {
              // float4 idx of the 64-byte-swizzled stage holds k-group g of its row
              const int idx = gt + r * kGen, row = idx >> 2, g = (idx & 3) ^ ((row >> 1) & 3);
              uint2 hi, lo;
              bf16_split4(v[r], hi, lo);
              *(uint2*)(Alo + swz32(row, g)) = hi;
              *(uint2*)(Alo + SA / 2 + swz32(row, g)) = lo;
            } else {
              float4 l;
              l.x = tf32_hi(v[r].x - tf32_trunc(v[r].x));
              l.y = tf32_hi(v[r].y - tf32_trunc(v[r].y));
              l.z = tf32_hi(v[r].z - tf32_trunc(v[r].z));
              l.w = tf32_hi(v[r].w - tf32_trunc(v[r].w));
              l4[gt + r * kGen] = l;
            }
          }
      }
#pragma unroll
      for (int r = 0; r < kItems; ++r) {
        const int row = it_row[r], kq = it_kq[r], i = row & 3;
        if (row >= NCP) continue;
        // k of this step within its half (uniform over the CTA: no step mixes the halves)
        const bool im = kc >= KH;
        const int kb = (im ? kc - KH : kc) * kKC + kq * 4;
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        if (fast) {
          const int npr = it_pb[r] - it_pa[r];
#pragma unroll
          for (int pp = 0; pp < 2; ++pp) {
            if (pp < npr) {
              const float4 cf = ycf[r][pp];
              const float4* ip = Ir + soff[r][pp] + kb;
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const float4 iv = ip[q];
                z[q] += cf.x * iv.x + cf.y * iv.y + cf.z * iv.z + cf.w * iv.w;
              }
            }
          }
        } else {
          for (int pl = it_pa[r]; pl < it_pb[r]; ++pl) {
            const float* y = y_in_smem ? Ysb + pl * 32 : p.Y + ((ybase + pl) * p.ntile + ti) * 32;
            const float4 ya = *(const float4*)(y + i * 8), yb = *(const float4*)(y + i * 8 + 4);
            const float4 cf = im ? make_float4(-ya.y, -ya.w, -yb.y, -yb.w) : make_float4(ya.x, ya.z, yb.x, yb.z);
            const int sl = (pl < kYPairs) ? pslot[pl] : -1;
            const float4* ir = reinterpret_cast<const float4*>(Icz) + (size_t)pair_in[pp0 + pl] * N;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int k = kb + q;
              if (sl < 0 && k >= N) continue;                 // padded column (zero in the staged slots)
              const float4 iv = sl >= 0 ? Ir[sl * IS + k] : ir[k];
              z[q] += cf.x * iv.x + cf.y * iv.y + cf.z * iv.z + cf.w * iv.w;
            }
          }
        }
        if constexpr (kBF16) {
          uint2 hi, lo;
          bf16_split4(make_float4(z[0], z[1], z[2], z[3]), hi, lo);
          *(uint2*)(Bhi + swz32(row, kq)) = hi;
          *(uint2*)(Blo + swz32(row, kq)) = lo;
        } else {
          float4 hi, lo;
          hi.x = tf32_hi(z[0]); lo.x = tf32_hi(z[0] - hi.x);
          hi.y = tf32_hi(z[1]); lo.y = tf32_hi(z[1] - hi.y);
          hi.z = tf32_hi(z[2]); lo.z = tf32_hi(z[2] - hi.z);
          hi.w = tf32_hi(z[3]); lo.w = tf32_hi(z[3] - hi.w);
          *(float4*)(Bhi + swz64(row, kq * 4)) = hi;
          *(float4*)(Blo + swz64(row, kq * 4)) = lo;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&ready[cb]);
    }
    // ---------------- epilogue: TMEM -> registers -> eps_bar
    // warp-uniform: the TMEM loads and the shuffles below need the whole warp
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0, abort_flag, p.spin));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int q = warp & 3;                    // TMEM lane quarter of this warp
      const int par = (warp - 2) >> 2;           // kGenWarps / 4 warps per quarter split the 16-column groups
      const int r = q * 32 + lane;               // D row: Stokes column (output el = r / 4, i = r % 4)
      const int si = lane & 3;                   // its Stokes index
      const bool live = r < 4 * E;
      const int o = live ? cout_dir[e0 + (r >> 2)] : 0;
      float* dst = p.eb + (((size_t)iz * p.nO + o) * N) * 4;
      for (int c0 = par * 16; c0 < NM; c0 += 16 * (kGenWarps / 4)) {
        uint32_t v[16];
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // The 4 lanes of an output hold its 4 Stokes values for the 16 columns; a 4 x 4
        // transpose per group of 4 columns (three exchanges) gives lane si the 4 Stokes
        // values of column 4m + si, added with one vector reduction instead of four.
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const float a0 = __uint_as_float(v[4 * m]), a1 = __uint_as_float(v[4 * m + 1]);
          const float a2 = __uint_as_float(v[4 * m + 2]), a3 = __uint_as_float(v[4 * m + 3]);
          auto pick = [&](int k) { return k == 0 ? a0 : (k == 1 ? a1 : (k == 2 ? a2 : a3)); };
          float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;   // Stokes 0..3 of column 4m + si
          auto put = [&](int k, float x) {
            if (k == 0) s0 = x;
            else if (k == 1) s1 = x;
            else if (k == 2) s2 = x;
            else s3 = x;
          };
          put(si, pick(si));
#pragma unroll
          for (int x = 1; x < 4; ++x) put(si ^ x, __shfl_xor_sync(0xffffffffu, pick(si ^ x), x));
          const int n = c0 + 4 * m + si;
          if (live && n < N)
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + (size_t)n * 4), "f"(s0),
                         "f"(s1), "f"(s2), "f"(s3)
                         : "memory");
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicExch(p.err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tm_cols));
  }
}

}  // namespace tc

// Tile stages for N rows: the most (<= kStagesMax) whose shared memory fits.
static int r2_tc_stages(int N, bool split) {
  for (int st = tc::kStagesMax; st >= 2; --st)
    if (tc::smem_bytes(N, st, split) <= tc::kSmemMax) return st;
  return 0;
}

// Work list and error flag of the tensor-core contraction.
int r2_tc_prepare(Ctx* c) {
  // the device error flag of the bounded waits (contraction and staged sweep), all precisions
  if (!c->tc_err.p) {
    int rc = dalloc(c, c->tc_err, sizeof(int));
    if (rc) return rc;
    PRD_CUDA_TRY(c, cudaMemset(c->tc_err.p, 0, sizeof(int)));
  }
  if (c->prec != PRD_FP32) return PRD_OK;
  if (!c->tiled() || r2_tc_stages(c->nnu, false) < 2)
    return fail(c, PRD_E_ARG, "tensor-core contraction needs FP32 tiles and N small enough for two tile stages "
                              "beside the resident I~ (N <= 224)");
  // work items: every class split into chunks of <= kMaxE output directions
  std::vector<int> work;
  for (int k = 0; k < c->ncls; ++k)
    for (int e = c->cout_ptr[k]; e < c->cout_ptr[k + 1]; e += tc::kMaxE) {
      work.push_back(k);
      work.push_back(e);
    }
  c->tc_nwork = (int)work.size() / 2;
  dfree(c->tc_work);
  {
    int rc = dalloc(c, c->tc_work, work.size() * sizeof(int));
    if (rc) return rc;
  }
  PRD_CUDA_TRY(c, cudaMemcpy(c->tc_work.p, work.data(), work.size() * sizeof(int), cudaMemcpyHostToDevice));
  PRD_CUDA_TRY(c, cudaMemset(c->tc_err.p, 0, sizeof(int)));
  c->tc_ready = true;
  return PRD_OK;
}

int r2_tc_launch(Ctx* c, const float* Ic, float* eb) {
  // the deepest ring that fits, or the caller's (autotuned) depth if smaller
  const int nmax = r2_tc_stages(c->nnu, c->split_tiles);
  const int nst = c->tc_stages >= 2 ? std::min(c->tc_stages, nmax) : nmax;
  tc::Params p{(const float*)c->tiles.p, (const float*)c->Y.p, Ic, (const int2*)c->tc_work.p,
               (const int*)c->cls_dev.p, eb, (int*)c->tc_err.p, c->ncls, c->ntile(), c->nO, c->nnu, c->npairs,
               c->ld(), nst, c->tc_spin > 0 ? c->tc_spin : tc::kSpin};
  const int smem = tc::smem_bytes(c->nnu, nst, c->split_tiles);
  auto go = [&](auto kern) -> int {
    PRD_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    kern<<<dim3(c->tc_nwork, c->nz), tc::kThreads, smem, c->stream>>>(p);
    return PRD_OK;
  };
  int rc;
  if (c->hi_only) rc = go(tc::r2_tc_kernel<true, true, true>);
  else if (c->split_tiles) rc = go(tc::r2_tc_kernel<true, true, false>);
  else if (c->tc_bf16) rc = go(tc::r2_tc_kernel<true, false, false>);
  else rc = go(tc::r2_tc_kernel<false, false, false>);
  if (rc) return rc;
  PRD_CUDA_TRY(c, cudaPeekAtLastError());
  return PRD_OK;
}

int r2_tc_check_error(Ctx* c) {
  int h = 0;
  PRD_CUDA_TRY(c, cudaMemcpy(&h, c->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    cudaMemset(c->tc_err.p, 0, sizeof(int));
    return fail(c, PRD_E_TIMEOUT, "tensor-core contraction: a bounded wait expired");
  }
  return PRD_OK;
}

}  // namespace prd
