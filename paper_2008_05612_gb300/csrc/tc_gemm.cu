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
//                     through a padded shared-memory square (coalesced rows), or a per-row
//                     running top-k; then arrive on tmem_empty[a].
// With two accumulators the epilogue of tile i overlaps the MMAs of tile i + 1.  Every mbarrier
// wait is bounded; one that gives up raises a shared abort flag (the other roles stop at their
// next wait) and the device error word, and each role drains what it has in flight before the
// CTA frees its tensor memory.
#include <cuda.h>

#include <algorithm>
#include <climits>
#include <cmath>
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
// 8 epilogue warps in both modes: two per tensor-memory lane quarter, 128 columns each (top-k
// mode also keeps its warp's 128 biases of the current tile in shared memory); a 3-stage ring
// leaves room for their shared-memory areas
template <int KT>
struct Shape {
  static constexpr int kEpiWarps = 4 * kTcListsPerTile;
  static constexpr int kThreads = 64 + 32 * kEpiWarps;
  static constexpr int kColsPerWarp = TN / (kEpiWarps / 4);
  static constexpr int kStages = 3;
  static constexpr int kAreaFloats = KT > 0 ? SX_FLOATS + kColsPerWarp : KT < 0 ? SQ_FLOATS + kColsPerWarp : SQ_FLOATS;
  static constexpr int kSmem = kStages * STAGE_BYTES + kEpiWarps * kAreaFloats * 4 + 1024;
};
constexpr uint32_t SPIN_LIMIT = 1u << 24;

// Work unit u: m tile u % mt and the column tiles [r nt / nr, (r + 1) nt / nr) of r = u / mt.
// Store mode uses one column tile per unit (nr = nt); top-k mode carries each row's list across
// the tiles of a unit, so its threshold rises early and few columns need an insertion.
// With split-K (store mode only) a unit is also one of ksplit slices of the K chunks.
struct Params {
  int M, N, K, mt, nt, nr, units, ksplit;
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
  const int r = rest / p.mt;
  return {(rest % p.mt) * TM,
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

// instruction descriptor: bf16 x bf16 -> f32, both K-major, M = 128, N = 256
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// four floats as four bf16 in one 8-byte store (dst 8-byte aligned)
__device__ __forceinline__ void store_bf16x4(bf16* dst, float a, float b, float c, float d) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  uint2 u;
  u.x = *reinterpret_cast<const uint32_t*>(&lo);
  u.y = *reinterpret_cast<const uint32_t*>(&hi);
  *reinterpret_cast<uint2*>(dst) = u;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%"
      "21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int KT>
__global__ void __launch_bounds__(Shape<KT>::kThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, const Params p) {
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
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
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
          tma_load(dst, &map_a, kc * TK, w.m0, fb);
          tma_load(dst + A_BYTES, &map_b, kc * TK, tn * TN, fb);
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
                "l"(desc(a_addr + ks * 32)), "l"(desc(b_addr + ks * 32)), "r"(IDESC), "r"(accumulate));
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
    float* area = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES) + (warp - 2) * Shape<KT>::kAreaFloats;
    float* bsm = area + (KT > 0 ? SX_FLOATS : SQ_FLOATS);  // top-k / softmax modes: this warp's biases of the tile
    const TcEpilogue& ep = p.ep;
    // top-k mode: biases of the next tile, one column per lane and 32-column chunk, loaded a
    // whole tile ahead of use
    float bnext[KT != 0 ? CW / 32 : 1];
    auto fetch_bias = [&](int n0) {
      if constexpr (KT != 0) {
#pragma unroll
        for (int i = 0; i < CW / 32; i++) {
          const int c = n0 + cbeg + 32 * i + lane;
          bnext[i] = (ep.bias && c < p.N) ? __ldg(ep.bias + c) : 0.f;
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
      if constexpr (KT == -2) {
        if (my_row < p.M) {
          rm = ep.row_m[my_row];
          rs = ep.row_inv[my_row];
        }
      }
      for (int tn = w.nb; tn < w.ne; tn++, tl++) {
        const uint32_t a = tl & 1, ar = tl >> 1;
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
            if (cl < p.N) {
              const int rmax = min(32, p.M - rbase);
              for (int r = 0; r < rmax; r++) {
                const size_t row = (size_t)(rbase + r);
                float x = area[r * 33 + lane] + bl;
                if (ep.relu) x = fmaxf(x, 0.f);
                if (ep.Cf) ep.Cf[(size_t)w.ks * ep.split_stride + row * ep.ldcf + cl] = x;
                if (ep.Cb) ep.Cb[row * ep.ldcb + cl] = __float2bfloat16(x);
              }
            }
            __syncwarp();
          } else if constexpr (KT < 0) {
            const int cmax = min(32, p.N - (n0 + c0));
            const int cbase = n0 + c0;
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              const float4 b4 = *reinterpret_cast<const float4*>(bsm + (c0 - cbeg) + j);
              v[j] = __float_as_uint(__uint_as_float(v[j]) + b4.x);
              v[j + 1] = __float_as_uint(__uint_as_float(v[j + 1]) + b4.y);
              v[j + 2] = __float_as_uint(__uint_as_float(v[j + 2]) + b4.z);
              v[j + 3] = __float_as_uint(__uint_as_float(v[j + 3]) + b4.w);
            }
            if constexpr (KT == -1) {
              // running max and sum of exponentials over the chunk's valid columns
              float cm = -INFINITY;
#pragma unroll
              for (int j = 0; j < 32; j++)
                if (j < cmax) cm = fmaxf(cm, __uint_as_float(v[j]));
              const float nm = fmaxf(rm, cm);
              float acc = 0.f;
#pragma unroll
              for (int j = 0; j < 32; j++)
                if (j < cmax) acc += __expf(__uint_as_float(v[j]) - nm);
              rs = (rm == -INFINITY ? 0.f : rs * __expf(rm - nm)) + acc;
              rm = nm;
              if (lab >= cbase && lab < cbase + cmax) {  // once per row: pick the label's logit
#pragma unroll
                for (int j = 0; j < 32; j++) area[lane * 33 + j] = __uint_as_float(v[j]);
                zl = area[lane * 33 + (lab - cbase)];
                have_zl = true;
              }
            } else {
              // dz = (softmax - onehot) * scale into the padded square (row = lane), then both
              // layouts are written from it: a full 32 x 32 block four bf16 per lane and store
              // (8-byte stores, 256 bytes per warp instruction), a ragged one element by element
#pragma unroll
              for (int j = 0; j < 32; j++) {
                const int col = cbase + j;
                float d = 0.f;
                if (lab >= 0 && j < cmax) d = (__expf(__uint_as_float(v[j]) - rm) * rs - (col == lab ? 1.f : 0.f)) * ep.scale;
                area[lane * 33 + j] = d;
              }
              __syncwarp();
              const int rmax = min(32, p.M - rbase);
              if (cmax == 32 && rmax == 32) {
                const int sub = lane >> 3, quad = (lane & 7) * 4;
#pragma unroll
                for (int r = 0; r < 32; r += 4) {
                  const float* a = area + (r + sub) * 33 + quad;  // row r + sub, columns quad .. + 3
                  store_bf16x4(ep.dz + (size_t)(rbase + r + sub) * ep.ldz + cbase + quad, a[0], a[1], a[2], a[3]);
                  const float* t = area + quad * 33 + (r + sub);  // column r + sub, rows quad .. + 3
                  store_bf16x4(ep.dzt + (size_t)(cbase + r + sub) * ep.ldzt + rbase + quad, t[0], t[33], t[66], t[99]);
                }
              } else {
                if (lane < cmax)
                  for (int r = 0; r < rmax; r++)
                    ep.dz[(size_t)(rbase + r) * ep.ldz + cbase + lane] = __float2bfloat16(area[r * 33 + lane]);
                if (lane < rmax)
                  for (int j = 0; j < cmax; j++)
                    ep.dzt[(size_t)(cbase + j) * ep.ldzt + rbase + lane] = __float2bfloat16(area[lane * 33 + j]);
              }
              __syncwarp();
            }
          } else {
            // 1. bias-added logits of the chunk
            const int cmax = min(32, p.N - (n0 + c0));
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              const float4 b4 = *reinterpret_cast<const float4*>(bsm + (c0 - cbeg) + j);
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
                  int ci = ep.col_id ? __ldg(ep.col_id + n0 + c0 + j) : n0 + c0 + j;
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
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(&tmem_empty[a])) : "memory");
      }
      if constexpr (KT == -1) {
        if (ok && my_row < p.M) {
          const size_t l = (size_t)(w.r * kTcListsPerTile + h);
          *reinterpret_cast<float2*>(ep.stats + 2 * (l * p.M + my_row)) = make_float2(rm, rs);
          if (have_zl) ep.zlab[my_row] = zl;
        }
      }
      if constexpr (KT > 0) {
        const int row = rbase + lane;
        if (ok && row < p.M) {
          // list l = 2 r + h of this row
          const size_t off = ((size_t)(w.r * kTcListsPerTile + h) * p.M + row) * KT;
#pragma unroll
          for (int j = 0; j < KT; j += 4) {
            *reinterpret_cast<float4*>(ep.cand_v + off + j) = make_float4(bv[j], bv[j + 1], bv[j + 2], bv[j + 3]);
            *reinterpret_cast<int4*>(ep.cand_i + off + j) = make_int4(bi[j], bi[j + 1], bi[j + 2], bi[j + 3]);
          }
        }
      }
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

// Per row: combine the (max, sum of exp) pairs of all lists.
__global__ void softmax_finish_kernel(const float* __restrict__ stats, int lists, int rows, const int32_t* __restrict__ labels,
                                      const float* __restrict__ zlab, float* __restrict__ row_m, float* __restrict__ row_inv,
                                      float* __restrict__ loss) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  float m = -INFINITY, s = 0.f;
  for (int l = 0; l < lists; l++) {
    const float2 q = *reinterpret_cast<const float2*>(stats + 2 * ((size_t)l * rows + r));
    if (q.x == -INFINITY) continue;
    const float nm = fmaxf(m, q.x);
    s = (m == -INFINITY ? 0.f : s * __expf(m - nm)) + q.y * __expf(q.x - nm);
    m = nm;
  }
  row_m[r] = m;
  row_inv[r] = 1.f / s;
  if (labels && labels[r] >= 0) atomicAdd(loss, logf(s) + m - zlab[r]);
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

// rows x K bf16, row stride ld elements; boxes of 64 (K) x box_rows, 128-byte swizzle, zero fill
int make_map(CUtensorMap* map, const bf16* base, int rows, int K, int ld, int box_rows) {
  EncodeTiled enc = encode_fn();
  if (!enc) return fail(HP_ECUDA, "tc_gemm: cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
  cuuint32_t elem[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(base), dims, strides, box, elem,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HP_EINVAL, "tc_gemm: tensor map rejected (alignment or stride)");
  return HP_OK;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

template <int KT>
void launch(const CUtensorMap& ma, const CUtensorMap& mb, const Params& p, cudaStream_t st) {
  cudaFuncSetAttribute(gemm_tc_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, Shape<KT>::kSmem);
  const int grid = std::min(p.units, sm_count());
  gemm_tc_kernel<KT><<<grid, Shape<KT>::kThreads, Shape<KT>::kSmem, st>>>(ma, mb, p);
}

}  // namespace

int tc_topk_lists(int M, int N) {
  // as many column ranges as make the units a multiple of the SM count (balanced waves), times
  // the two column slices of each tile (one list per epilogue warp)
  const int mt = (M + TM - 1) / TM, nt = (N + TN - 1) / TN, g = sm_count();
  return std::max(1, std::min(nt, g / std::gcd(mt, g))) * kTcListsPerTile;
}

int tc_gemm(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, const TcEpilogue& ep, unsigned* err,
            cudaStream_t st) {
  if (M < 1 || N < 1 || K < 1 || lda % 8 || ldb % 8 || lda < K || ldb < K ||
      (reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) % 16)
    return fail(HP_EINVAL, "tc_gemm: bad shape, stride or alignment");
  if (ep.kt > 0 && ((ep.kt != 4 && ep.kt != 8 && ep.kt != 16) || !ep.cand_v || !ep.cand_i))
    return fail(HP_EINVAL, "tc_gemm: top-k mode needs kt in {4, 8, 16} and candidate buffers");
  if (ep.kt == -1 && (!ep.stats || !ep.zlab || !ep.labels))
    return fail(HP_EINVAL, "tc_gemm: row-statistics mode needs stats, zlab and labels");
  if (ep.kt == -2 && (!ep.row_m || !ep.row_inv || !ep.labels || !ep.dz || !ep.dzt || (ep.ldz | ep.ldzt) <= 0))
    return fail(HP_EINVAL, "tc_gemm: gradient mode needs row statistics, labels and both outputs");
  if (ep.kt < -2) return fail(HP_EINVAL, "tc_gemm: unknown epilogue mode");
  CUtensorMap ma, mb;
  int rc = make_map(&ma, A, M, K, lda, TM);
  if (rc == HP_OK) rc = make_map(&mb, B, N, K, ldb, TN);
  if (rc != HP_OK) return rc;
  const int nk = (K + TK - 1) / TK;
  if (ep.ksplit < 1 || ep.ksplit > nk || (ep.ksplit > 1 && (ep.kt || ep.Cb || ep.bias || ep.relu || !ep.Cf)))
    return fail(HP_EINVAL, "tc_gemm: split-K needs store mode with an fp32 output only and at most one slice per K chunk");
  Params p{M, N, K, (M + TM - 1) / TM, (N + TN - 1) / TN, 0, 0, ep.ksplit, ep, err,
           (uint32_t)std::min<long long>(wait_limit(SPIN_LIMIT), 0xFFFFFFFFll)};
  p.nr = (ep.kt > 0 || ep.kt == -1) ? tc_topk_lists(M, N) / kTcListsPerTile : p.nt;
  p.units = p.mt * p.nr * p.ksplit;
  switch (ep.kt) {
    case 0: launch<0>(ma, mb, p, st); break;
    case -1: launch<-1>(ma, mb, p, st); break;
    case -2: launch<-2>(ma, mb, p, st); break;
    case 4: launch<4>(ma, mb, p, st); break;
    case 8: launch<8>(ma, mb, p, st); break;
    default: launch<16>(ma, mb, p, st); break;
  }
  return HP_OK;
}

void tc_softmax_finish(const float* stats, int lists, int rows, const int32_t* labels, const float* zlab, float* row_m,
                       float* row_inv, float* loss, cudaStream_t st) {
  softmax_finish_kernel<<<(rows + 255) / 256, 256, 0, st>>>(stats, lists, rows, labels, zlab, row_m, row_inv, loss);
}

void tc_topk_merge(const float* cand_v, const int32_t* cand_i, int tiles, int rows, int kt, int k, int S, int32_t* out,
                   cudaStream_t st) {
  const dim3 block(256), grid((rows + 7) / 8);
  if (kt == 4) topk_merge_kernel<4><<<grid, block, 0, st>>>(cand_v, cand_i, tiles, rows, k, S, out);
  else if (kt == 8) topk_merge_kernel<8><<<grid, block, 0, st>>>(cand_v, cand_i, tiles, rows, k, S, out);
  else topk_merge_kernel<16><<<grid, block, 0, st>>>(cand_v, cand_i, tiles, rows, k, S, out);
}

}  // namespace hp
