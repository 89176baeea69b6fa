// tcgen05 GEMM for the proposal network (see tc_gemm.h).
//
// One persistent CTA per SM walks the 128 x 256 output tiles (m fastest, so the CTAs running at
// the same time share B tiles in L2).  Warp roles:
//   warp 0, one lane  TMA producer: 64-wide K chunks of A (128 x 64) and B (256 x 64) into a
//                     3-stage ring, 128-byte swizzled, completion counted on full[s];
//   warp 1, one lane  MMA issuer: four tcgen05.mma (M 128, N 256, K 16) per chunk into one of two
//                     tensor-memory accumulators (2 x 256 columns), commit -> empty[s] frees the
//                     stage, commit -> tmem_full[a] hands the finished accumulator over;
//   warps 2..9        epilogue, two warps per lane quarter and 128 columns each: tcgen05.ld
//                     (warp w reads lanes 32 (w % 4) .. +31 = tile rows), bias, ReLU, stores
//                     through a padded shared-memory square (coalesced rows), a per-row
//                     running top-k, or the softmax statistics or gradient (the gradient's
//                     32 x 32 blocks leave through TMA stores); then arrive on tmem_empty[a].
// With two accumulators the epilogue of tile i overlaps the MMAs of tile i + 1.  Every mbarrier
// wait is bounded; one that gives up raises a shared abort flag (the other roles stop at their
// next wait) and the device error word, and each role drains what it has in flight before the
// CTA frees its tensor memory.
#include <cuda.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>

#include "hp_internal.h"
#include "tc_gemm.h"

namespace hp {
namespace {

using bf16 = __nv_bfloat16;

constexpr int TM = kTcTileM, TN = kTcTileN, TK = 64;
constexpr int A_BYTES = TM * TK * 2, B_BYTES = TN * TK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SQ_FLOATS = 32 * 33;  // store mode: one epilogue warp's padded 32 x 32 square
constexpr int SX_FLOATS = 32 * 32;  // top-k mode: one epilogue warp's staged logits (XOR-swizzled rows)
// gradient mode: per epilogue warp two staging buffers, each a 32 x 32 bf16 block of dz
// (row-major, 64-byte rows), the sources of the TMA stores
constexpr int STG_BLOCK = 32 * 32 * 2, STG_WARP = 2 * STG_BLOCK;
// Epilogue warps: 16, four per tensor-memory lane quarter, 64 columns each (more warps hide the
// tensor-memory and global-memory latencies of the epilogues), except in top-k mode, which keeps
// 8 (two per lane quarter, 128 columns each; each warp keeps one candidate list per row).  Top-k and
// softmax modes also keep the warp's biases of the current tile in shared memory; a 3-stage ring
// leaves room for the warps' shared-memory areas.
template <int KT>
struct Shape {
  static constexpr int kEpiWarps = KT > 0 ? 4 * tc_topk_lists_per_tile(KT) : 16;
  static constexpr int kThreads = 64 + 32 * kEpiWarps;
  static constexpr int kColsPerWarp = TN / (kEpiWarps / 4);
  static constexpr int kStages = 3;
  static constexpr int kAreaFloats = KT > 0 ? SX_FLOATS + kColsPerWarp : KT < 0 ? kColsPerWarp : SQ_FLOATS;
  static constexpr int kStgBytes = KT == -2 ? kEpiWarps * STG_WARP : 0;
  static constexpr int kSmem = kStages * STAGE_BYTES + kStgBytes + kEpiWarps * kAreaFloats * 4 + 1024;
};
constexpr uint32_t SPIN_LIMIT = 1u << 24;

// Work unit u: m tile u % mt and the column tiles [r nt / nr, (r + 1) nt / nr) of r = u / mt
// (with nfast, r = u % nr and m tile u / nr).  Store mode uses one column tile per unit (nr = nt)
// and nfast when A is the larger operand, so that the CTAs running at the same time share A tiles
// in L2; top-k mode carries each row's list across the tiles of a unit, so its threshold rises
// early and few columns need an insertion.  With split-K (store mode only) a unit is also one of
// ksplit slices of the K chunks (the slices of one tile are neighbouring units).
struct Params {
  int M, N, K, mt, nt, nr, units, ksplit, nfast;
  int a_mn, b_mn;  // operand stored MN-major ([K][M] / [K][N]) instead of K-major
  TcEpilogue ep;
  unsigned* err;
  uint32_t spin;  // polls of a pipeline wait before it gives up (the exit drains keep SPIN_LIMIT)
};

struct Unit {
  int m0, nb, ne, r, ks, kb, ke;  // ks: K slice; [kb, ke): its K chunks
};

__device__ __forceinline__ Unit unit_of(const Params& p, int u) {
  const int nk = (p.K + TK - 1) / TK;
  const int ks = u % p.ksplit, rest = u / p.ksplit;
  const int r = p.nfast ? rest % p.nr : rest / p.mt;
  return {(p.nfast ? rest / p.nr : rest % p.mt) * TM,
          (int)((long long)r * p.nt / p.nr),
          (int)((long long)(r + 1) * p.nt / p.nr),
          r,
          ks,
          (int)((long long)ks * nk / p.ksplit),
          (int)((long long)(ks + 1) * nk / p.ksplit)};
}

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool poll(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok)
               : "r"(bar), "r"(parity)
               : "memory");
  return ok != 0;
}

// Wait for the phase of `bar` with this parity.  False if another role aborted (checked every
// 256 polls) or, after `limit` polls, this one gives up (then it raises the abort flag and the
// error word); a limit of 0 gives up before the first poll.
__device__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag, unsigned* err, uint32_t limit) {
  const uint32_t b = sa(bar);
  for (uint32_t i = 0;; i++) {
    if (i >= limit) {
      *abort_flag = 1;
      if (err) atomicOr(err, 1u);
      return false;
    }
    if (poll(b, parity)) return true;
    if ((i & 255) == 255 && *abort_flag) return false;
  }
}

// Drain wait used on the way out: bounded, not cut short by the abort flag.
__device__ void drain(uint64_t* bar, uint32_t parity, unsigned* err) {
  const uint32_t b = sa(bar);
  for (uint32_t i = 0; i < SPIN_LIMIT; i++)
    if (poll(b, parity)) return;
  if (err) atomicOr(err, 2u);
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1 KB apart
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}

// shared-memory matrix descriptor: MN-major, 128-byte swizzle: 8 K rows of 64 MN elements
// (128 bytes each) form a 1 KB atom; K groups of 8 rows 1 KB apart (stride offset), blocks of
// 64 MN elements 8 KB apart (leading offset: one TMA box of 64 x 64 each)
__device__ __forceinline__ uint64_t desc_mn(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(8192 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor: bf16 x bf16 -> f32, both K-major, M = 128, N = 256 (bits 15 / 16 make
// A / B MN-major)
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
constexpr int MN_BOX = 64;  // MN-major operands: TMA boxes of 64 MN elements x TK K rows (8 KB)

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// 32 lanes x 32 columns of tensor memory into v, issued only: tmem_wait(v) makes them usable
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%"
      "21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

// wait for the issued tensor-memory loads; v is tied to the wait so that no use of it is
// scheduled before it
__device__ __forceinline__ void tmem_wait(uint32_t (&v)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]),
                 "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]),
                 "+r"(v[23]), "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]),
                 "+r"(v[30]), "+r"(v[31])
               :
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  tmem_ld32_issue(taddr, v);
  tmem_wait(v);
}

// two floats as bf16 (round to nearest even), lo in the low half
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 t = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&t);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Row-statistics chunk (one row per lane, 32 columns): the logits are acc + bias; the running max
// rm and sum rs of exp(logit - rm) take the chunk's first cmax columns, and the logit at column
// lab_rel (if in range) goes to zl
__device__ __forceinline__ void stats_chunk(const uint32_t (&acc)[32], const float* bias, int cmax, int lab_rel, float& rm,
                                            float& rs, float& zl, bool& have_zl) {
  constexpr float kLog2e = 1.4426950408889634f;
  float x[32];
#pragma unroll
  for (int j = 0; j < 32; j += 4) {
    const float4 b4 = *reinterpret_cast<const float4*>(bias + j);
    x[j] = __uint_as_float(acc[j]) + b4.x;
    x[j + 1] = __uint_as_float(acc[j + 1]) + b4.y;
    x[j + 2] = __uint_as_float(acc[j + 2]) + b4.z;
    x[j + 3] = __uint_as_float(acc[j + 3]) + b4.w;
  }
  float cm = -INFINITY;
#pragma unroll
  for (int j = 0; j < 32; j++)
    if (j < cmax) cm = fmaxf(cm, x[j]);
  const float nm = fmaxf(rm, cm), nml = nm * kLog2e;
  float sum = 0.f;
#pragma unroll
  for (int j = 0; j < 32; j++)
    if (j < cmax) sum += ex2_approx(fmaf(x[j], kLog2e, -nml));
  rs = (rm == -INFINITY ? 0.f : rs * ex2_approx((rm - nm) * kLog2e)) + sum;
  rm = nm;
  if (lab_rel >= 0 && lab_rel < cmax) {
#pragma unroll
    for (int j = 0; j < 32; j++)
      if (j == lab_rel) zl = x[j];
    have_zl = true;
  }
}

// Byte offset of byte b (0..63) of row r in a 32 x 32 bf16 staging block with the TMA's 64-byte
// swizzle: the 16-byte chunk b / 16 of a 64-byte row is stored at chunk (b / 16) ^ ((r / 2) % 4),
// so that 8 consecutive rows writing the same chunk hit 8 different bank groups (the block is
// 512-byte aligned)
__device__ __forceinline__ uint32_t stg_off(int r, int b) {
  return (uint32_t)(r * 64 + ((((b >> 4) ^ (r >> 1)) & 3) << 4) + (b & 15));
}

// Top-k chunk (one row per lane, 32 columns): the logits acc + bias enter the row's running list
// (bv, bi: value descending, index ascending) if they reach its last entry; the first full chunk
// seeds the threshold with the smallest of KT group maxima.  Warp-collective.
template <int KT>
__device__ __forceinline__ void topk_chunk(uint32_t (&v)[32], const float* bias, int cmax, int colbase,
                                           const int32_t* col_id, float (&bv)[KT], int (&bi)[KT], bool& seeded,
                                           float* area, int lane) {
  // 1. bias-added logits of the chunk (cmax of its columns are valid)
#pragma unroll
  for (int j = 0; j < 32; j += 4) {
    const float4 b4 = *reinterpret_cast<const float4*>(bias + j);
    v[j] = __float_as_uint(__uint_as_float(v[j]) + b4.x);
    v[j + 1] = __float_as_uint(__uint_as_float(v[j + 1]) + b4.y);
    v[j + 2] = __float_as_uint(__uint_as_float(v[j + 2]) + b4.z);
    v[j + 3] = __float_as_uint(__uint_as_float(v[j + 3]) + b4.w);
  }
  // 2. the columns that can enter: at least the list's current last (equal values are
  //    settled on their ids below) or, for the list's first full chunk, at least the
  //    smallest of KT group maxima (KT columns reach it, so nothing below it is among
  //    the KT best)
  float thr = nextafterf(bv[KT - 1], -INFINITY);  // x > thr  <=>  x >= last
  if (!seeded && cmax == 32) {
    constexpr int G = 32 / KT;
    float t0 = INFINITY;
#pragma unroll
    for (int g = 0; g < KT; g++) {
      float mg = __uint_as_float(v[g * G]);
#pragma unroll
      for (int e = 1; e < G; e++) mg = fmaxf(mg, __uint_as_float(v[g * G + e]));
      t0 = fminf(t0, mg);
    }
    thr = nextafterf(t0, -INFINITY);  // x > thr  <=>  x >= t0
    seeded = true;
  }
  uint32_t part[8];
#pragma unroll
  for (int g = 0; g < 8; g++) {
    uint32_t m4 = 0;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const float x = __uint_as_float(v[4 * g + e]);
      m4 |= (uint32_t)(x > thr) << e;
    }
    part[g] = m4 << (4 * g);
  }
  uint32_t mask = ((part[0] | part[1]) | (part[2] | part[3])) | ((part[4] | part[5]) | (part[6] | part[7]));
  if (cmax < 32) mask &= (1u << cmax) - 1u;
  if (__any_sync(0xFFFFFFFFu, mask != 0)) {
    // 3. stage the row (16-byte groups XOR-swizzled by lane: conflict-free), then
    //    insert each lane's candidates in column order, one per lane per round
#pragma unroll
    for (int g = 0; g < 8; g++)
      *reinterpret_cast<uint4*>(area + lane * 32 + ((g ^ (lane & 7)) << 2)) =
          make_uint4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
    __syncwarp();
    while (__any_sync(0xFFFFFFFFu, mask != 0)) {
      if (mask) {
        const int j = __ffs(mask) - 1;
        mask &= mask - 1;
        float cv = area[lane * 32 + (((j >> 2) ^ (lane & 7)) << 2) + (j & 3)];
        int ci = col_id ? __ldg(col_id + colbase + j) : colbase + j;
        if (cv > bv[KT - 1] || (cv == bv[KT - 1] && ci < bi[KT - 1])) {
#pragma unroll
          for (int e = 0; e < KT; e++) {
            const bool take = cv > bv[e] || (cv == bv[e] && ci < bi[e]);
            const float tv = bv[e];
            const int ti = bi[e];
            bv[e] = take ? cv : bv[e];
            bi[e] = take ? ci : bi[e];
            cv = take ? tv : cv;
            ci = take ? ti : ci;
          }
        }
      }
    }
    __syncwarp();
  }
}

// TMA store of a 32 x 32 bf16 box from shared memory at tensor coordinates (x, y); the part of
// the box outside the tensor is not written
__device__ __forceinline__ void tma_store(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map), "r"(src), "r"(x),
               "r"(y)
               : "memory");
}

template <int KT>
__global__ void __launch_bounds__(Shape<KT>::kThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                   const __grid_constant__ CUtensorMap map_dz, const Params p) {
  constexpr int STAGES = Shape<KT>::kStages;
  extern __shared__ uint8_t tc_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], tmem_full[2], tmem_empty[2], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_word;
  volatile int* abort_flag = &abort_word;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(sa(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&empty[s])));
    }
    for (int a = 0; a < 2; a++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&tmem_full[a])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(&tmem_empty[a])), "r"(32 * Shape<KT>::kEpiWarps));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&done)));
    abort_word = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&map_a) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&map_b) : "memory");
    if constexpr (KT == -2) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&map_dz) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // the set-up above touched no global memory; everything below may read the previous kernel's
  // results
  pdl_wait();
  pdl_trigger();
  const uint32_t tmem = tmem_base;
  unsigned* err = p.err;

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------------- TMA producer
    uint32_t it = 0;  // chunks issued; chunk it goes to stage it % STAGES, round it / STAGES
    bool ok = true;
    for (int u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
      const Unit w = unit_of(p, u);
      for (int tn = w.nb; tn < w.ne && ok; tn++) {
        for (int kc = w.kb; kc < w.ke; kc++, it++) {
          const uint32_t s = it % STAGES, r = it / STAGES;
          // round r reuses the stage after the MMAs of round r - 1 committed (round 0: fresh barrier)
          if (!wait_or_abort(&empty[s], (r & 1) ^ 1, abort_flag, err, p.spin)) {
            ok = false;
            break;
          }
          const uint32_t fb = sa(&full[s]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(STAGE_BYTES) : "memory");
          const uint32_t dst = sa(smem + s * STAGE_BYTES);
          if (p.a_mn) {
            for (int j = 0; j < TM / MN_BOX; j++) tma_load(dst + j * MN_BOX * TK * 2, &map_a, w.m0 + j * MN_BOX, kc * TK, fb);
          } else {
            tma_load(dst, &map_a, kc * TK, w.m0, fb);
          }
          if (p.b_mn) {
            for (int j = 0; j < TN / MN_BOX; j++)
              tma_load(dst + A_BYTES + j * MN_BOX * TK * 2, &map_b, tn * TN + j * MN_BOX, kc * TK, fb);
          } else {
            tma_load(dst + A_BYTES, &map_b, kc * TK, tn * TN, fb);
          }
        }
      }
    }
    // every load issued has landed before the CTA may exit
    for (uint32_t s = 0; s < STAGES; s++) {
      const uint32_t cnt = it > s ? (it - s + STAGES - 1) / STAGES : 0;
      if (cnt) drain(&full[s], (cnt - 1) & 1, err);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------------- MMA issuer
    uint32_t it = 0, tl = 0;
    bool ok = true;
    const uint32_t idesc = IDESC | ((uint32_t)(p.a_mn != 0) << 15) | ((uint32_t)(p.b_mn != 0) << 16);
    for (int u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
      const Unit w = unit_of(p, u);
      for (int tn = w.nb; tn < w.ne && ok; tn++, tl++) {
        const uint32_t a = tl & 1, ar = tl >> 1;
        if (!wait_or_abort(&tmem_empty[a], (ar & 1) ^ 1, abort_flag, err, p.spin)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_addr = tmem + a * TN;
        for (int kc = w.kb; kc < w.ke; kc++, it++) {
          const uint32_t s = it % STAGES, r = it / STAGES;
          if (!wait_or_abort(&full[s], r & 1, abort_flag, err, p.spin)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a_addr = sa(smem + s * STAGE_BYTES), b_addr = a_addr + A_BYTES;
#pragma unroll
          for (int ks = 0; ks < TK / 16; ks++) {
            const uint32_t accumulate = (kc != w.kb || ks != 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                    acc_addr),
                "l"(p.a_mn ? desc_mn(a_addr + ks * 2048) : desc(a_addr + ks * 32)),
                "l"(p.b_mn ? desc_mn(b_addr + ks * 2048) : desc(b_addr + ks * 32)), "r"(idesc), "r"(accumulate));
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(&empty[s]))
                       : "memory");
        }
        if (ok)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           sa(&tmem_full[a]))
                       : "memory");
      }
    }
    // all MMAs issued by this thread complete, and every stage release has arrived
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(&done)) : "memory");
    drain(&done, 0, err);
    for (uint32_t s = 0; s < STAGES; s++) {
      const uint32_t cnt = it > s ? (it - s + STAGES - 1) / STAGES : 0;
      if (cnt) drain(&empty[s], (cnt - 1) & 1, err);
    }
  } else if (warp >= 2) {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3;                          // tensor-memory lane quarter this warp may read
    const int h = (warp - 2) >> 2;                   // which column slice of each tile
    constexpr int CW = Shape<KT>::kColsPerWarp;
    const int cbeg = h * CW, cend = cbeg + CW;
    float* area = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES + Shape<KT>::kStgBytes) + (warp - 2) * Shape<KT>::kAreaFloats;
    // top-k / softmax modes: this warp's biases of the tile
    float* bsm = area + (KT > 0 ? SX_FLOATS : 0);
    // gradient mode: this warp's staging buffers and the count of blocks it has staged
    uint8_t* stg = smem + STAGES * STAGE_BYTES + (warp - 2) * STG_WARP;
    uint32_t staged = 0;
    const TcEpilogue& ep = p.ep;
    // top-k mode: biases of the next tile, one column per lane and 32-column chunk, loaded a
    // whole tile ahead of use
    float bnext[KT != 0 ? CW / 32 : 1];
    auto fetch_bias = [&](int n0) {
      if constexpr (KT != 0) {
#pragma unroll
        for (int i = 0; i < CW / 32; i++) {
          const int c = n0 + cbeg + 32 * i + lane;
          // (gradient mode keeps the biases scaled by log2 e)
          bnext[i] = (ep.bias && c < p.N) ? __ldg(ep.bias + c) * (KT == -2 ? 1.4426950408889634f : 1.f) : 0.f;
        }
      }
    };
    if (KT != 0 && (int)blockIdx.x < p.units) fetch_bias(unit_of(p, blockIdx.x).nb * TN);
    uint32_t tl = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
      const Unit w = unit_of(p, u);
      const int rbase = w.m0 + q * 32;  // first row of this warp
      // top-k mode: one running list per row over this warp's columns of all tiles of the unit,
      // ordered by (value descending, id ascending)
      float bv[KT > 0 ? KT : 1];
      int bi[KT > 0 ? KT : 1];
#pragma unroll
      for (int j = 0; j < (KT > 0 ? KT : 1); j++) {
        bv[j] = -INFINITY;
        bi[j] = INT_MAX;
      }
      bool seeded = false;
      // softmax modes: this thread's row, its label and (statistics) running max / sum or
      // (gradient) the row's max and 1 / sum
      const int my_row = rbase + lane;
      const int lab = (KT < 0 && my_row < p.M && ep.labels) ? ep.labels[my_row] : -1;
      float rm = -INFINITY, rs = 0.f, zl = 0.f;
      bool have_zl = false;
      // gradient mode, with the logit x = acc + bias and t = acc log2 e + bias log2 e:
      //   dz = exp2(t + kc) rss (kc = -m log2 e, rss = scale / sum; rss = 0 for a row without
      //   label), or, when every row of the warp has |m| < 64 (no overflow), dz = exp2(t) rss2
      //   with rss2 = rss exp2(kc); the label's entry, (exp(x_label - m) / sum - 1) scale from the
      //   label logit of the statistics pass, replaces the staged value of its column
      float kc = 0.f, rss = 0.f, rss2 = 0.f, dlab = 0.f;
      bool fast = true;
      if constexpr (KT == -2) {
        constexpr float kLog2e = 1.4426950408889634f;
        if (my_row < p.M) {
          const float m = ep.row_m[my_row];
          kc = -m * kLog2e;
          fast = fabsf(m) < 64.f;
          if (lab >= 0) {
            rss = ep.row_inv[my_row] * ep.scale;
            dlab = fmaf(ex2_approx(fmaf(ep.zlab[my_row], kLog2e, kc)), rss, -ep.scale);
          }
          rss2 = rss * ex2_approx(kc);
        }
        fast = __all_sync(0xFFFFFFFFu, fast);
      }
      for (int tn = w.nb; tn < w.ne; tn++, tl++) {
        const uint32_t a = tl & 1, ar = tl >> 1;
        // store mode with a ReLU mask: bit r of keepm[i] says whether row rbase + r of this lane's
        // column in chunk i is kept; loaded while the tile's MMAs run
        uint32_t keepm[KT == 0 ? CW / 32 : 1];
        if constexpr (KT == 0) {
          const int rmax = min(32, p.M - rbase);
#pragma unroll
          for (int i = 0; i < CW / 32; i++) {
            const int cl = tn * TN + cbeg + 32 * i + lane;
            uint32_t keep = ~0u;
            if (ep.relu_mask && cl < p.N) {
              keep = 0u;
#pragma unroll
              for (int r = 0; r < 32; r++)
                if (r < rmax && __bfloat162float(__ldg(ep.relu_mask + (size_t)(rbase + r) * ep.ldmask + cl)) > 0.f)
                  keep |= 1u << r;
            }
            keepm[i] = keep;
          }
        }
        if (!wait_or_abort(&tmem_full[a], ar & 1, abort_flag, err, p.spin)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int n0 = tn * TN;
        if constexpr (KT != 0) {
          __syncwarp();
#pragma unroll
          for (int i = 0; i < CW / 32; i++) bsm[32 * i + lane] = bnext[i];
          const int nt_next = tn + 1 < w.ne ? tn + 1 : (u + (int)gridDim.x < p.units ? unit_of(p, u + gridDim.x).nb : -1);
          if (nt_next >= 0) fetch_bias(nt_next * TN);
          __syncwarp();
        }
        if constexpr (KT < 0) {
          // ---- softmax modes, one 32-column chunk at a time (the 16 epilogue warps hide the
          // tensor-memory latency).  Row statistics: running max and sum of exponentials over the
          // chunk's valid columns, and the label's logit.  Gradient: dz, staged as a bf16 block
          // (row-major) and stored by TMA; the block's column sums go to colpart.
          const uint32_t tbase = tmem + a * TN + ((uint32_t)(q * 32) << 16) + (uint32_t)cbeg;
          const int nch = min(CW / 32, (p.N - n0 - cbeg + 31) / 32);  // chunks holding columns < N
#pragma unroll 1
          for (int i = 0; i < nch; i++) {
            uint32_t v[32];
            __syncwarp();
            tmem_ld32(tbase + 32 * i, v);
            const int c0 = cbeg + 32 * i, cbase = n0 + c0;
            if constexpr (KT == -1) {
              stats_chunk(v, bsm + 32 * i, min(32, p.N - cbase), lab - cbase, rm, rs, zl, have_zl);
            } else {
              // dz in place (as float bits)
#pragma unroll
              for (int j = 0; j < 32; j += 4) {
                const float4 b4 = *reinterpret_cast<const float4*>(bsm + (c0 - cbeg) + j);
                const float bj[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                  const float t = fmaf(__uint_as_float(v[j + e]), 1.4426950408889634f, bj[e]);
                  v[j + e] = __float_as_uint(fast ? ex2_approx(t) * rss2 : ex2_approx(t + kc) * rss);
                }
              }
              // this buffer's previous TMA store has read it (at most the other buffer's pending)
              uint8_t* buf = stg + (staged & 1) * STG_BLOCK;
              if (staged >= 2 && lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
              __syncwarp();
              // row-major block (swizzled): lane = row, 64 bytes; then the label's entry of this
              // row, if its column is in the chunk
              {
#pragma unroll
                for (int k = 0; k < 4; k++)
                  *reinterpret_cast<uint4*>(buf + stg_off(lane, 16 * k)) = make_uint4(pack_bf16(__uint_as_float(v[8 * k]), __uint_as_float(v[8 * k + 1])),
                                      pack_bf16(__uint_as_float(v[8 * k + 2]), __uint_as_float(v[8 * k + 3])),
                                      pack_bf16(__uint_as_float(v[8 * k + 4]), __uint_as_float(v[8 * k + 5])),
                                      pack_bf16(__uint_as_float(v[8 * k + 6]), __uint_as_float(v[8 * k + 7])));
                const int lr = lab - cbase;
                if (lab >= 0 && lr >= 0 && lr < 32)
                  *reinterpret_cast<__nv_bfloat16*>(buf + stg_off(lane, lr * 2)) = __float2bfloat16(dlab);
              }
              asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
              __syncwarp();
              if (rbase < p.M) {
                if (ep.colpart) {
                  // column sums of the stored values: lane l adds the column pair l % 16 over the
                  // 16 rows of half l / 16 (the upper half visits its rows in a shifted order, so
                  // that the two halves never share a bank), then the halves are added
                  const int cp = lane & 15, rh = lane >> 4;
                  float s0 = 0.f, s1 = 0.f;
#pragma unroll
                  for (int k = 0; k < 16; k++) {
                    const int r = 16 * rh + (k ^ rh);
                    const uint32_t wv = *reinterpret_cast<const uint32_t*>(buf + stg_off(r, cp * 4));
                    s0 += __uint_as_float(wv << 16);
                    s1 += __uint_as_float(wv & 0xFFFF0000u);
                  }
                  s0 += __shfl_xor_sync(0xFFFFFFFFu, s0, 16);
                  s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, 16);
                  const int c = cbase + 2 * cp + rh;  // lanes < 16 write the even, the others the odd column
                  if (c < p.N) ep.colpart[(size_t)(rbase >> 5) * p.N + c] = rh ? s1 : s0;
                }
                if (lane == 0) {
                  tma_store(&map_dz, sa(buf), cbase, rbase);
                  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                }
              }
              staged++;
            }
          }
        } else if constexpr (KT > 0) {
          // ---- top-k: chunks alternate between two register sets, the next one's tensor-memory
          // load in flight while the current one is filtered
          const uint32_t tbase = tmem + a * TN + ((uint32_t)(q * 32) << 16) + (uint32_t)cbeg;
          const int nch = min(CW / 32, (p.N - n0 - cbeg + 31) / 32);
          uint32_t va[32], vb[32];
          __syncwarp();
          if (nch > 0) tmem_ld32(tbase, va);
#pragma unroll 1
          for (int i = 0; i < nch; i += 2) {
            if (i + 1 < nch) tmem_ld32_issue(tbase + 32 * (i + 1), vb);
            topk_chunk<KT>(va, bsm + 32 * i, min(32, p.N - (n0 + cbeg + 32 * i)), n0 + cbeg + 32 * i, ep.col_id, bv, bi,
                           seeded, area, lane);
            if (i + 1 < nch) {
              tmem_wait(vb);
              if (i + 2 < nch) tmem_ld32_issue(tbase + 32 * (i + 2), va);
              topk_chunk<KT>(vb, bsm + 32 * (i + 1), min(32, p.N - (n0 + cbeg + 32 * (i + 1))), n0 + cbeg + 32 * (i + 1),
                             ep.col_id, bv, bi, seeded, area, lane);
              if (i + 2 < nch) tmem_wait(va);
            }
          }
        } else {
#pragma unroll 1
          for (int c0 = cbeg; c0 < cend && n0 + c0 < p.N; c0 += 32) {
            uint32_t v[32];
            __syncwarp();  // tcgen05.ld is warp-collective
            tmem_ld32(tmem + a * TN + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
            if constexpr (KT == 0) {
              const int cl = n0 + c0 + lane;  // this lane's column
              const float bl = (ep.bias && cl < p.N) ? ep.bias[cl] : 0.f;
#pragma unroll
              for (int j = 0; j < 32; j++) area[lane * 33 + j] = __uint_as_float(v[j]);
              __syncwarp();
              const int rmax = min(32, p.M - rbase);
              if (ep.adam_w) {
                // Adam step on the gradient chunk: the weights and moments of its rows are loaded
                // together, then updated; the new weights go back into the square for the
                // transposed copy
                // (8 rows at a time: 24 loads in flight per lane)
                for (int h16 = 0; h16 < 32 && cl < p.N; h16 += 8) {
                  float w32[8], m32[8], v32[8];
#pragma unroll
                  for (int e = 0; e < 8; e++) {
                    const int r = h16 + e;
                    const size_t i = (size_t)(rbase + r) * ep.ldcf + cl;
                    w32[e] = r < rmax ? ep.adam_w[i] : 0.f;
                    m32[e] = r < rmax ? ep.adam_m[i] : 0.f;
                    v32[e] = r < rmax ? ep.adam_v[i] : 0.f;
                  }
#pragma unroll
                  for (int e = 0; e < 8; e++) {
                    const int r = h16 + e;
                    if (r < rmax) {
                      const size_t row = (size_t)(rbase + r), i = row * ep.ldcf + cl;
                      const float g = area[r * 33 + lane];
                      const float mi = ep.b1 * m32[e] + (1.f - ep.b1) * g;
                      const float vi = ep.b2 * v32[e] + (1.f - ep.b2) * g * g;
                      // Kingma & Ba's update; fast division, IEEE square root
                      const float wi = w32[e] - __fdividef(ep.lr * (mi * ep.c1), __fsqrt_rn(vi * ep.c2) + ep.eps);
                      ep.adam_m[i] = mi;
                      ep.adam_v[i] = vi;
                      ep.adam_w[i] = wi;
                      if (ep.Cb) ep.Cb[row * ep.ldcb + cl] = __float2bfloat16(wi);
                      area[r * 33 + lane] = wi;
                    }
                  }
                }
                __syncwarp();
                if (ep.wt && lane < rmax) {
                  const int cmax = min(32, p.N - (n0 + c0));
                  for (int j = 0; j < cmax; j++)
                    ep.wt[(size_t)(n0 + c0 + j) * ep.ldwt + rbase + lane] = __float2bfloat16(area[lane * 33 + j]);
                }
              } else if (cl < p.N) {
                uint32_t keep = keepm[0];  // this chunk's mask bits (~0 without a mask)
#pragma unroll
                for (int i = 1; i < CW / 32; i++)
                  if (c0 - cbeg == 32 * i) keep = keepm[i];
                for (int r = 0; r < rmax; r++) {
                  const size_t row = (size_t)(rbase + r);
                  float x = area[r * 33 + lane] + bl;
                  if (ep.relu) x = fmaxf(x, 0.f);
                  if (!((keep >> r) & 1u)) x = 0.f;
                  if (ep.Cf) ep.Cf[(size_t)w.ks * ep.split_stride + row * ep.ldcf + cl] = x;
                  if (ep.Cb) ep.Cb[row * ep.ldcb + cl] = __float2bfloat16(x);
                }
              }
              __syncwarp();
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(&tmem_empty[a])) : "memory");
      }
      if constexpr (KT == -1) {
        if (ok && my_row < p.M) {
          static_assert(Shape<KT>::kEpiWarps / 4 == kTcStatsListsPerTile, "one statistics list per column slice");
          const size_t l = (size_t)(w.r * kTcStatsListsPerTile + h);
          *reinterpret_cast<float2*>(ep.stats + 2 * (l * p.M + my_row)) = make_float2(rm, rs);
          if (have_zl) ep.zlab[my_row] = zl;
        }
      }
      if constexpr (KT > 0) {
        const int row = rbase + lane;
        if (ok && row < p.M) {
          // list l = 2 r + h of this row
          const size_t off = ((size_t)(w.r * tc_topk_lists_per_tile(KT) + h) * p.M + row) * KT;
#pragma unroll
          for (int j = 0; j < KT; j += 4) {
            *reinterpret_cast<float4*>(ep.cand_v + off + j) = make_float4(bv[j], bv[j + 1], bv[j + 2], bv[j + 3]);
            *reinterpret_cast<int4*>(ep.cand_i + off + j) = make_int4(bi[j], bi[j + 1], bi[j + 2], bi[j + 3]);
          }
        }
      }
    }
    // gradient mode: every TMA store of this warp has completed before the CTA exits
    if constexpr (KT == -2) {
      if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// Per row (one warp), the k best of `lists` sorted candidate lists of KT: each lane merges the
// lists lane, lane + 32, ... into its own list ordered by (value descending, index ascending);
// then k shuffle rounds pick the best head across the warp.
template <int KT>
__global__ void topk_merge_kernel(const float* __restrict__ cv, const int32_t* __restrict__ ci, int tiles, int rows, int k,
                                  int S, int32_t* __restrict__ out) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  float bv[KT];
  int bi[KT];
#pragma unroll
  for (int j = 0; j < KT; j++) {
    bv[j] = -INFINITY;
    bi[j] = INT_MAX;
  }
  for (int t = lane; t < tiles; t += 32) {
    const size_t off = ((size_t)t * rows + row) * KT;
#pragma unroll
    for (int j = 0; j < KT; j++) {
      float v = cv[off + j];
      int i = ci[off + j];
      // lists cover interleaved column sets, so compare (value, index); a list is sorted, so
      // once an entry does not enter, no later entry of the same list does
      if (!(v > bv[KT - 1] || (v == bv[KT - 1] && i < bi[KT - 1]))) break;
#pragma unroll
      for (int u = 0; u < KT; u++) {
        const bool take = v > bv[u] || (v == bv[u] && i < bi[u]);
        const float tv = bv[u];
        const int ti = bi[u];
        bv[u] = take ? v : bv[u];
        bi[u] = take ? i : bi[u];
        v = take ? tv : v;
        i = take ? ti : i;
      }
    }
  }
  for (int r = 0; r < k; r++) {
    float v = bv[0];
    int i = bi[0];
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      const float ov = __shfl_xor_sync(0xFFFFFFFFu, v, off);
      const int oi = __shfl_xor_sync(0xFFFFFFFFu, i, off);
      if (ov > v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
      }
    }
    if (lane == 0) out[(size_t)row * k + r] = i < S ? i : -1;
    if (bi[0] == i && i != INT_MAX) {  // the winning lane pops its head
#pragma unroll
      for (int j = 0; j < KT - 1; j++) {
        bv[j] = bv[j + 1];
        bi[j] = bi[j + 1];
      }
      bv[KT - 1] = -INFINITY;
      bi[KT - 1] = INT_MAX;
    }
  }
}

// Per row (one warp, lanes over the lists): combine the (max, sum of exp) pairs of all lists.
__global__ void softmax_finish_kernel(const float* __restrict__ stats, int lists, int rows, const int32_t* __restrict__ labels,
                                      const float* __restrict__ zlab, float* __restrict__ row_m, float* __restrict__ row_inv,
                                      float* __restrict__ loss) {
  pdl_wait();
  pdl_trigger();
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const bool row_ok = r < rows;  // whole warps past the last row still meet the block barrier below
  float m = -INFINITY, s = 0.f;
  for (int l = lane; row_ok && l < lists; l += 32) {
    const float2 q = *reinterpret_cast<const float2*>(stats + 2 * ((size_t)l * rows + r));
    if (q.x == -INFINITY) continue;
    const float nm = fmaxf(m, q.x);
    s = (m == -INFINITY ? 0.f : s * __expf(m - nm)) + q.y * __expf(q.x - nm);
    m = nm;
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    const float om = __shfl_xor_sync(0xFFFFFFFFu, m, off), os = __shfl_xor_sync(0xFFFFFFFFu, s, off);
    const float nm = fmaxf(m, om);
    if (nm != -INFINITY) s = (m == -INFINITY ? 0.f : s * __expf(m - nm)) + (om == -INFINITY ? 0.f : os * __expf(om - nm));
    m = nm;
  }
  if (lane == 0 && row_ok) {
    row_m[r] = m;
    row_inv[r] = 1.f / s;
  }
  // the rows' cross-entropies: summed over the block's rows, one atomic add per block (a single
  // address takes every add)
  __shared__ float part[32];
  if (lane == 0) part[threadIdx.x >> 5] = (row_ok && labels && labels[r] >= 0) ? logf(s) + m - zlab[r] : 0.f;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
    if (labels && t != 0.f) atomicAdd(loss, t);
  }
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                                const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
  });
  return fn;
}

// An operand of `rows` (M or N) x K bf16: K-major ([rows][K], row stride ld) in boxes of 64 (K) x
// box_rows, or MN-major ([K][rows], row stride ld) in boxes of 64 (rows) x 64 (K); 128-byte
// swizzle, zero fill outside the operand
int make_map(CUtensorMap* map, const bf16* base, int rows, int K, int ld, int box_rows, bool mn_major) {
  EncodeTiled enc = encode_fn();
  if (!enc) return fail(HP_ECUDA, "tc_gemm: cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[2] = {(cuuint64_t)(mn_major ? rows : K), (cuuint64_t)(mn_major ? K : rows)};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)(mn_major ? TK : box_rows)};
  cuuint32_t elem[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(base), dims, strides, box, elem,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HP_EINVAL, "tc_gemm: tensor map rejected (alignment or stride)");
  return HP_OK;
}

// rows x cols bf16 (row stride ld elements) as the destination of 32 x 32 TMA stores; the shared
// memory source uses the 64-byte swizzle (see stg_off)
int make_store_map(CUtensorMap* map, const bf16* base, int rows, int cols, int ld) {
  EncodeTiled enc = encode_fn();
  if (!enc) return fail(HP_ECUDA, "tc_gemm: cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t elem[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(base), dims, strides, box, elem,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HP_EINVAL, "tc_gemm: output tensor map rejected (alignment or stride)");
  return HP_OK;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

template <int KT>
void launch(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mdz, const Params& p, cudaStream_t st) {
  static_assert(Shape<KT>::kSmem <= 227 * 1024, "shared memory of the tcgen05 GEMM");
  cudaFuncSetAttribute(gemm_tc_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, Shape<KT>::kSmem);
  const int grid = std::min(p.units, sm_count());
  launch_pdl(gemm_tc_kernel<KT>, dim3(grid), dim3(Shape<KT>::kThreads), Shape<KT>::kSmem, st, ma, mb, mdz, p);
}

}  // namespace

// column ranges of the top-k and statistics modes: as many as make the units a multiple of the
// SM count (balanced waves)
int tc_ranges(int M, int N) {
  const int mt = (M + TM - 1) / TM, nt = (N + TN - 1) / TN, g = sm_count();
  return std::max(1, std::min(nt, g / std::gcd(mt, g)));
}

int tc_stats_lists(int M, int N) { return tc_ranges(M, N) * kTcStatsListsPerTile; }

int tc_topk_lists(int M, int N, int kt) { return tc_ranges(M, N) * tc_topk_lists_per_tile(kt); }


int tc_gemm(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, const TcEpilogue& ep, unsigned* err,
            cudaStream_t st) {
  if (M < 1 || N < 1 || K < 1 || lda % 8 || ldb % 8 || lda < (ep.a_mn ? M : K) || ldb < (ep.b_mn ? N : K) ||
      (reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) % 16)
    return fail(HP_EINVAL, "tc_gemm: bad shape, stride or alignment");
  if (ep.kt > 0 && ((ep.kt != 4 && ep.kt != 8 && ep.kt != 16) || !ep.cand_v || !ep.cand_i))
    return fail(HP_EINVAL, "tc_gemm: top-k mode needs kt in {4, 8, 16} and candidate buffers");
  if (ep.kt == -1 && (!ep.stats || !ep.zlab || !ep.labels))
    return fail(HP_EINVAL, "tc_gemm: row-statistics mode needs stats, zlab and labels");
  if (ep.kt == -2 && (!ep.row_m || !ep.row_inv || !ep.labels || !ep.zlab || !ep.dz || ep.ldz < N || ep.ldz % 8 ||
                      reinterpret_cast<uintptr_t>(ep.dz) % 16))
    return fail(HP_EINVAL, "tc_gemm: gradient mode needs row statistics, labels and dz (strides a multiple of 8, 16-byte aligned)");
  if (ep.kt < -2) return fail(HP_EINVAL, "tc_gemm: unknown epilogue mode");
  if (ep.relu_mask && (ep.kt || ep.adam_w || ep.ksplit != 1 || ep.ldmask < N))
    return fail(HP_EINVAL, "tc_gemm: the ReLU-mask epilogue takes a plain store-mode GEMM");
  if (ep.adam_w && (ep.kt || ep.Cf || ep.bias || ep.relu || ep.ksplit != 1 || !ep.adam_m || !ep.adam_v || ep.ldcf < N ||
                    (ep.wt && ep.ldwt < M)))
    return fail(HP_EINVAL, "tc_gemm: the Adam epilogue takes a plain store-mode GEMM and its moment buffers");
  CUtensorMap ma, mb, mdz;
  memset(&mdz, 0, sizeof(mdz));
  int rc = make_map(&ma, A, M, K, lda, TM, ep.a_mn);
  if (rc == HP_OK) rc = make_map(&mb, B, N, K, ldb, TN, ep.b_mn);
  if (rc == HP_OK && ep.kt == -2) rc = make_store_map(&mdz, ep.dz, M, N, ep.ldz);
  if (rc != HP_OK) return rc;
  const int nk = (K + TK - 1) / TK;
  if (ep.ksplit < 1 || ep.ksplit > nk || (ep.ksplit > 1 && (ep.kt || ep.Cb || ep.bias || ep.relu || !ep.Cf)))
    return fail(HP_EINVAL, "tc_gemm: split-K needs store mode with an fp32 output only and at most one slice per K chunk");
  Params p{M, N, K, (M + TM - 1) / TM, (N + TN - 1) / TN, 0, 0, ep.ksplit, 0, ep.a_mn ? 1 : 0, ep.b_mn ? 1 : 0, ep, err,
           (uint32_t)std::min<long long>(wait_limit(SPIN_LIMIT), 0xFFFFFFFFll)};
  p.nr = (ep.kt > 0 || ep.kt == -1) ? tc_ranges(M, N) : p.nt;
  p.nfast = ep.kt == 0 && M > N;
  p.units = p.mt * p.nr * p.ksplit;
  switch (ep.kt) {
    case 0: launch<0>(ma, mb, mdz, p, st); break;
    case -1: launch<-1>(ma, mb, mdz, p, st); break;
    case -2: launch<-2>(ma, mb, mdz, p, st); break;
    case 4: launch<4>(ma, mb, mdz, p, st); break;
    case 8: launch<8>(ma, mb, mdz, p, st); break;
    default: launch<16>(ma, mb, mdz, p, st); break;
  }
  return HP_OK;
}

void tc_softmax_finish(const float* stats, int lists, int rows, const int32_t* labels, const float* zlab, float* row_m,
                       float* row_inv, float* loss, cudaStream_t st) {
  launch_pdl(softmax_finish_kernel, dim3((rows + 7) / 8), dim3(256), 0, st, stats, lists, rows, labels, zlab, row_m, row_inv,
             loss);
}

void tc_topk_merge(const float* cand_v, const int32_t* cand_i, int tiles, int rows, int kt, int k, int S, int32_t* out,
                   cudaStream_t st) {
  const dim3 block(256), grid((rows + 7) / 8);
  if (kt == 4) topk_merge_kernel<4><<<grid, block, 0, st>>>(cand_v, cand_i, tiles, rows, k, S, out);
  else if (kt == 8) topk_merge_kernel<8><<<grid, block, 0, st>>>(cand_v, cand_i, tiles, rows, k, S, out);
  else topk_merge_kernel<16><<<grid, block, 0, st>>>(cand_v, cand_i, tiles, rows, k, S, out);
}

}  // namespace hp
