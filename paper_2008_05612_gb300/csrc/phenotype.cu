// Ground-state phenotype kernel for sm_103a (Section 2.1 and Appendix C of
// arXiv 2008.05612: for every sequence, the conformation of lowest Eq. 1
// energy if it is unique, else -1).
//
// Arithmetic.  Write the score of sequence h on conformation s as
//   x_s(h) = -E_s(h) = sum over contacts (i, j) of 10 h_i + 10 h_j + 3 h_i h_j
// (Table 1 x 10: HH 23, HP 10, PP 0).  Consecutive residues sit on sites of
// opposite colour of the bipartite square/cubic lattice, so every contact joins
// an even residue to an odd one.  For a fixed pattern o of the odd residues the
// score is therefore AFFINE in the even residues e:
//   x_s(o, e) = base_s(o) + sum_{even k} e_k a_{s,k}(o),
//   base_s(o) = 10 sum_{odd j} o_j c_j(s),
//   a_{s,k}(o) = 10 c_{2k}(s) + 3 #{odd contact partners of residue 2k that are H in o}
// with c the per-residue contact counts.  One CTA owns one odd pattern o and
// 2^14 even patterns; the coefficients of each conformation are computed once
// per CTA and the scores of all even patterns are subset sums of them.
//
// Layout of the 14 even-pattern bits ("roles") for a shape with R register bits:
//   role 0            split: low/high 16-bit half of a packed register
//   roles 1..R-1      tree: index of one of the 2^(R-1) packed registers
//   roles R..R+4      lane of the warp
//   roles R+5..13     warp of the CTA (2^(9-R) warps)
// Each thread keeps, per packed register, the running maximum of the doubled,
// biased score 2 (x + 1) of two sequences (max.u16x2; the last tree level uses
// the fused add + max).  Per tile of T conformations the tile maximum is merged
// into a best value with a tie bit and the index of the first tile reaching it.
// A sequence whose best is reached in two tiles is not unique.  Pass 2 stages
// the tiles again and resolves every other sequence exactly inside its one tile
// (warp-cooperative count and first index with ballots), which also yields the
// lowest-index conformation at the minimum; each thread keeps a bit mask of its
// unresolved candidates, so it only reads those fields.
//
// Data movement.  Conformation records (contact masks, see hp_internal.h) are
// staged tile by tile into shared memory with the bulk-copy engine
// (cp.async.bulk + mbarrier, bounded waits), double buffered; one thread per
// conformation turns a record into the CTA's coefficient record (lane table,
// warp table, packed tree coefficients) in a second double buffer; in pass 1 the
// records of tile t + 1 are produced halfway through the consumption of tile t,
// and instead of a CTA barrier per tile the producer warps arrive on a "produced"
// mbarrier per buffer and every warp on a "consumed" one, so each warp waits only
// for the buffer it needs next (bounded waits).  CTAs are
// persistent and take work items (instance, id block, odd pattern, even chunk)
// from a device counter, so boxes of different shapes share one launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <new>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "hp_internal.h"
#include "phenotype.h"

namespace {

constexpr int kLaneRoles = 5;
constexpr int kRoles = 14;  // even-pattern bits covered by one CTA
constexpr unsigned kErrTimeout = 1u;
constexpr unsigned kErrDrain = 2u;  // the exit drain gave up with bulk copies in flight
constexpr long long kSpinLimit = 1ll << 26;  // polls of the exit drain (fixed); the other waits take PhenParams::spin

__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Wait for phase `parity` of the barrier; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit = kSpinLimit) {
  for (long long i = 0; i < limit; i++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// compressed even / odd bits of a sequence id (bit k = residue 2k / 2k+1)
__device__ __forceinline__ uint32_t even_bits(unsigned long long g) {
  uint32_t r = 0;
#pragma unroll
  for (int k = 0; k < hp::kMaxHalf; k++) r |= (uint32_t)((g >> (2 * k)) & 1ull) << k;
  return r;
}
__device__ __forceinline__ uint32_t odd_bits(unsigned long long g) {
  uint32_t r = 0;
#pragma unroll
  for (int k = 0; k < hp::kMaxHalf; k++) r |= (uint32_t)((g >> (2 * k + 1)) & 1ull) << k;
  return r;
}
__device__ __forceinline__ unsigned long long interleave(uint32_t e, uint32_t o) {
  unsigned long long g = 0;
#pragma unroll
  for (int k = 0; k < hp::kMaxHalf; k++)
    g |= ((unsigned long long)((e >> k) & 1u) << (2 * k)) | ((unsigned long long)((o >> k) & 1u) << (2 * k + 1));
  return g;
}

// coefficient of even residue 2k for odd pattern o: 10 c_{2k} + 3 #H partners
__device__ __forceinline__ uint32_t coef(uint32_t mask, uint32_t o) { return 10u * __popc(mask) + 3u * __popc(mask & o); }
// score part that depends on the odd residues only: 10 sum_j o_j c_j
__device__ __forceinline__ uint32_t odd_part(const uint32_t* r, int NE, uint32_t o) {
  return 10u * (__popc(o & r[NE]) + 2u * __popc(o & r[NE + 1]) + 4u * __popc(o & r[NE + 2]));
}

// Compile-time shape: R register bits (2^(R-1) packed registers of two
// sequences per thread), T conformations per shared-memory tile, ROLES even-pattern bits per CTA
// (14, or fewer for boxes and ranges with fewer free even residues), 2^(ROLES-5-R) warps.
template <int R_, int T_, int ROLES_ = kRoles>
struct Cfg {
  static constexpr int R = R_, T = T_, ROLES = ROLES_, WB = ROLES_ - kLaneRoles - R_;
  static constexpr int P = 1 << (R - 1);
  static constexpr int NW = 1 << WB;
  static constexpr int THREADS = 32 * NW;
  // coefficient record: lane table [32], warp table [NW], tree coefficients [R-1]
  static constexpr int WT_OFF = 32;
  static constexpr int TP_OFF = 32 + NW;
  static constexpr int TP_WORDS = ((R - 1) + 3) / 4 * 4;
  static constexpr int CS_RAW = TP_OFF + TP_WORDS;
  // words per record: a multiple of 4 that is odd in 16-byte units (conflict-free 16-byte stores)
  static constexpr int CSTRIDE = ((CS_RAW / 4) % 2 == 1) ? CS_RAW : CS_RAW + 4;
  // pass 2 reads word j of 32 consecutive records (one per lane): an odd stride in words keeps
  // those loads conflict-free, and the records are written with 4-byte stores
  static constexpr int CS2 = CS_RAW | 1;
  static constexpr int kCoefWords = 2 * T * (CSTRIDE > CS2 ? CSTRIDE : CS2);
  static constexpr int kStateWords = 2 * P * THREADS;
  static_assert(T <= THREADS, "one producer thread per conformation of a tile");
  static_assert(T % 32 == 0 && hp::kRecPad % T == 0, "tiles are whole warps and tile the padded table");
  static_assert(NW >= 4, "warp tables are written in groups of four");
};

// Turn the staged records of tile `tile` (the t-th tile of this pass; its bulk copy was issued two
// tiles ahead into raw buffer t & 1) into this CTA's coefficient records in buffer t & 1: one
// thread per conformation.  P2: the pass-2 layout (stride CS2, 4-byte stores) instead of pass 1's
// (stride CSTRIDE, 16-byte stores).  No barrier: the caller publishes the records (mbarrier
// arrive); a bounded wait that gives up raises *s_abort.
template <class K, bool P2 = false>
__device__ __forceinline__ void produce_work(const hp::PhenInst& in, unsigned* err, int t, int tile, uint32_t* rawbuf,
                                             uint32_t* coefbuf, uint64_t* bars,
                                             unsigned (&waited)[2], uint32_t o, uint32_t ehigh, int nroles,
                                             int* s_abort, long long spin) {
  constexpr int R = K::R, T = K::T;
  const int tid = threadIdx.x;
  const int buf = t & 1;
  constexpr int STRIDE = P2 ? K::CS2 : K::CSTRIDE;
  uint32_t* cbuf = coefbuf + buf * T * STRIDE;
  if (tid < T) {
    if (!mbar_wait(&bars[buf], waited[buf] & 1u, spin)) {
      atomicOr(err, kErrTimeout);
      *s_abort = 1;
    } else {
      const uint32_t* r = rawbuf + buf * T * in.rec_words + tid * in.rec_words;
      uint32_t* c = cbuf + tid * STRIDE;
      const int s = tile * T + tid;
      if (s < in.S_dir) {
        uint32_t a[K::ROLES];
#pragma unroll
        for (int k = 0; k < K::ROLES; k++) a[k] = k < nroles ? 2u * coef(r[k], o) : 0u;
        uint32_t extra = 0;
        for (int k = nroles; k < in.NE; k++)
          if ((ehigh >> k) & 1u) extra += coef(r[k], o);
        const uint32_t base = 2u * (odd_part(r, in.NE, o) + extra + 1u);
        const uint32_t split_hi = a[0] << 16;
        // lane table: base + subset sums of the 5 lane coefficients, packed
        uint32_t lt[32];
        lt[0] = base;
#pragma unroll
        for (int l = 1; l < 32; l++) {
          const int hb = 31 - __clz(l);
          lt[l] = lt[l ^ (1 << hb)] + a[R + hb];
        }
        if (P2) {
#pragma unroll
          for (int l = 0; l < 32; l++) c[l] = lt[l] * 0x10001u + split_hi;
        } else {
#pragma unroll
          for (int l = 0; l < 32; l += 4)
            *reinterpret_cast<uint4*>(c + l) = make_uint4(lt[l] * 0x10001u + split_hi, lt[l + 1] * 0x10001u + split_hi,
                                                          lt[l + 2] * 0x10001u + split_hi, lt[l + 3] * 0x10001u + split_hi);
        }
        uint32_t wt[K::NW];
        wt[0] = 0;
#pragma unroll
        for (int w = 1; w < K::NW; w++) {
          const int hb = 31 - __clz(w);
          wt[w] = wt[w ^ (1 << hb)] + a[R + kLaneRoles + hb];
        }
        uint32_t tp[K::TP_WORDS];
#pragma unroll
        for (int j = 0; j < K::TP_WORDS; j++) tp[j] = j < R - 1 ? a[1 + j] * 0x10001u : 0u;
        if (P2) {
#pragma unroll
          for (int w = 0; w < K::NW; w++) c[K::WT_OFF + w] = wt[w] * 0x10001u;
#pragma unroll
          for (int j = 0; j < R - 1; j++) c[K::TP_OFF + j] = tp[j];
        } else {
#pragma unroll
          for (int w = 0; w < K::NW; w += 4)
            *reinterpret_cast<uint4*>(c + K::WT_OFF + w) =
                make_uint4(wt[w] * 0x10001u, wt[w + 1] * 0x10001u, wt[w + 2] * 0x10001u, wt[w + 3] * 0x10001u);
#pragma unroll
          for (int j = 0; j < K::TP_WORDS; j += 4)
            *reinterpret_cast<uint4*>(c + K::TP_OFF + j) = make_uint4(tp[j], tp[j + 1], tp[j + 2], tp[j + 3]);
        }
      } else {
        // padding conformation: every score 0, below every real (biased) score
        if (P2) {
#pragma unroll
          for (int k = 0; k < K::CS_RAW; k++) c[k] = 0u;
        } else {
#pragma unroll
          for (int k = 0; k < K::CS_RAW; k += 4) *reinterpret_cast<uint4*>(c + k) = make_uint4(0, 0, 0, 0);
        }
      }
    }
  }
  waited[buf]++;
}

// Bulk copies of the first two tiles of a pass (tiles t0 and t1; t1 < 0: the pass has one tile).
template <int T>
__device__ __forceinline__ void prefetch_first_tiles(const hp::PhenInst& in, uint32_t* rawbuf, uint64_t* bars,
                                                     unsigned (&issued)[2], int t0, int t1) {
  const unsigned raw_bytes = (unsigned)(T * in.rec_words * 4);
  if (threadIdx.x == 0) bulk_load(rawbuf, in.rec + (size_t)t0 * T * in.rec_words, raw_bytes, &bars[0]);
  issued[0]++;
  if (t1 >= 0) {
    if (threadIdx.x == 0) bulk_load(rawbuf + T * in.rec_words, in.rec + (size_t)t1 * T * in.rec_words, raw_bytes, &bars[1]);
    issued[1]++;
  }
}

// GAP: energy-gap threshold above 1 (p.gap2 = 2 T in the doubled score units): pass 1 also keeps,
// per field, the largest tile maximum outside the first tile reaching the best (in the state area,
// unused during pass 1), and pass 2 counts the best tile's conformations within T of the best.
template <class K, bool GAP>
__global__ void __launch_bounds__(K::THREADS, 1) phenotype_kernel(const __grid_constant__ hp::PhenParams p) {
  constexpr int R = K::R, T = K::T, P = K::P, kThreads = K::THREADS, CSTRIDE = K::CSTRIDE;
  extern __shared__ __align__(128) uint32_t smem[];
  // layout: [coef 2 x T x CSTRIDE][raw 2 x T x max_rec_words][state 2 x P x THREADS][6 mbarriers:
  // raw copies (2), coefficient buffer produced (2), coefficient buffer consumed (2)]
  uint32_t* coefbuf = smem;
  uint32_t* rawbuf = smem + K::kCoefWords;
  uint32_t* st_best = rawbuf + 2 * T * p.max_rec_words;  // [P][THREADS] packed best (doubled score | tie)
  uint32_t* st_tile = st_best + P * kThreads;             // [P][THREADS] packed tile of the best, then result
  uint64_t* bars = reinterpret_cast<uint64_t*>(st_tile + P * kThreads);
  __shared__ int s_abort;
  __shared__ unsigned long long s_item;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], T / 32);      // one arrival per producer warp
    mbar_init(&bars[3], T / 32);
    mbar_init(&bars[4], kThreads / 32);  // one arrival per warp
    mbar_init(&bars[5], kThreads / 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  __syncthreads();
  // per raw buffer: bulk copies issued and waited for (identical in every thread)
  unsigned issued[2] = {0u, 0u}, waited[2] = {0u, 0u};
  // per coefficient buffer: productions waited for, and consumptions arrived (identical in every thread)
  unsigned fcnt0 = 0u, fcnt1 = 0u, ccnt0 = 0u, ccnt1 = 0u;
  const uint32_t role_hi = ((uint32_t)lane << R) | ((uint32_t)warp << (R + kLaneRoles));

  for (;;) {
    if (tid == 0) s_item = atomicAdd(reinterpret_cast<unsigned long long*>(p.ctrl + 2), 1ull);
    __syncthreads();
    const unsigned long long item = s_item;
    __syncthreads();  // s_item is rewritten by the next iteration
    if (item >= p.total_items) break;
    int b = 0;
    while (b + 1 < p.nblocks && p.blocks[b + 1].item_begin <= item) b++;
    const hp::PhenBlock& bd = p.blocks[b];
    const hp::PhenInst& in = p.inst[bd.inst];
    const unsigned long long local = item - bd.item_begin;
    uint32_t o, chunk;
    if (bd.otab) {
      o = bd.otab[local % bd.ntab];
      chunk = (uint32_t)(local / bd.ntab);
    } else {
      o = odd_bits(bd.g_base) | (uint32_t)(local & ((1ull << bd.no_free) - 1));
      chunk = (uint32_t)(local >> bd.no_free);
    }
    const int nroles = (int)bd.nroles;
    const uint32_t ehigh = even_bits(bd.g_base) | (chunk << nroles);
    const uint32_t role_mask = (1u << nroles) - 1u;
    const bool want_aux = in.aux != nullptr;

    // ================= pass 1: running maxima over every conformation
    uint32_t tmax[P], m1[P], ts[P];
#pragma unroll
    for (int v = 0; v < P; v++) tmax[v] = m1[v] = ts[v] = 0u;
    if (GAP)
      for (int v = 0; v < P; v++) st_best[v * kThreads + tid] = 0u;  // 0: no other tile yet
    prefetch_first_tiles<T>(in, rawbuf, bars, issued, 0, in.ntiles > 1 ? 1 : -1);
    // coefficient records of tile t + 1 are produced halfway through the consumption of tile t
    // (double buffered).  No CTA barrier: the producer warps arrive on full[b] when a buffer is
    // written, every warp arrives on empty[b] when it has consumed it, and a warp waits only for
    // the buffer it needs next, so fast warps run ahead instead of idling at a barrier.
    const bool producer = tid < T;
    // the tp-th tile of the pass, `tile` (pass 1: every tile, tile = tp; pass 2: the listed ones)
    auto produce_and_publish = [&](int tp, int tile, auto p2) {
      const int b = tp & 1;
      if (producer) {
        // the previous contents of buffer b (tile tp - 2) must have been consumed by every warp
        if (tp >= 2 && !mbar_wait(&bars[4 + b], ((b ? ccnt1 : ccnt0) - 1u) & 1u, p.spin_handover)) {
          atomicOr(p.ctrl, kErrTimeout);
          s_abort = 1;
        }
      }
      produce_work<K, decltype(p2)::value>(in, p.ctrl, tp, tile, rawbuf, coefbuf, bars, waited, o, ehigh, nroles,
                                           &s_abort, p.spin);
      if (producer) {
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bars[2 + b])) : "memory");
      }
    };
    using Pass1Layout = std::false_type;
    using Pass2Layout = std::true_type;
    produce_and_publish(0, 0, Pass1Layout{});
    for (int t = 0; t < in.ntiles; t++) {
      const int b = t & 1;
      if (!mbar_wait(&bars[2 + b], (b ? fcnt1 : fcnt0) & 1u, p.spin_handover)) {
        atomicOr(p.ctrl, kErrTimeout);
        s_abort = 1;
      }
      if (b) fcnt1++;
      else fcnt0++;
      if (s_abort) break;
      // every producer has read raw[b] (tile t): refill it with tile t + 2
      if (t + 2 < in.ntiles) {
        if (tid == 0)
          bulk_load(rawbuf + b * T * in.rec_words, in.rec + (size_t)(t + 2) * T * in.rec_words,
                    (unsigned)(T * in.rec_words * 4), &bars[b]);
        issued[b]++;
      }
      const uint32_t* cbuf = coefbuf + b * T * CSTRIDE;
      // subset sums over the tree roles of one conformation (IMAD: x * one + a keeps them on the FMA
      // pipe); the leaves (top tree bit set) are left to the fused add + max
      auto tree = [&](const uint32_t* cs, uint32_t (&x)[P / 2], uint32_t (&tpv)[K::TP_WORDS]) {
#pragma unroll
        for (int j = 0; j < K::TP_WORDS; j += 4) {
          const uint4 q = *reinterpret_cast<const uint4*>(cs + K::TP_OFF + j);
          tpv[j] = q.x; tpv[j + 1] = q.y; tpv[j + 2] = q.z; tpv[j + 3] = q.w;
        }
        x[0] = cs[lane] * p.one + cs[K::WT_OFF + warp];
#pragma unroll
        for (int v = 1; v < P / 2; v++) {
          const int hb = 31 - __clz(v);
          x[v] = x[v ^ (1 << hb)] * p.one + tpv[hb];
        }
      };
      auto consume = [&](int s0, int s1) {
        if constexpr (P <= 16) {
          // two conformations at a time: the lower half of the registers takes both with one
          // three-input packed max, the upper half with two fused add + max
#pragma unroll 8
          for (int s = s0; s < s1; s += 2) {
            uint32_t x[P / 2], y[P / 2], tx[K::TP_WORDS], ty[K::TP_WORDS];
            tree(cbuf + s * CSTRIDE, x, tx);
            tree(cbuf + (s + 1) * CSTRIDE, y, ty);
#pragma unroll
            for (int v = 0; v < P / 2; v++) {
              tmax[v] = __vimax3_u16x2(tmax[v], x[v], y[v]);
              tmax[v + P / 2] = __viaddmax_u16x2(y[v], ty[R - 2], __viaddmax_u16x2(x[v], tx[R - 2], tmax[v + P / 2]));
            }
          }
        } else {
#pragma unroll 8
          for (int s = s0; s < s1; s++) {
            uint32_t x[P / 2], tx[K::TP_WORDS];
            tree(cbuf + s * CSTRIDE, x, tx);
#pragma unroll
            for (int v = 0; v < P / 2; v++) {
              tmax[v] = vmax2(tmax[v], x[v]);
              tmax[v + P / 2] = __viaddmax_u16x2(x[v], tx[R - 2], tmax[v + P / 2]);
            }
          }
        }
      };
      consume(0, T / 2);
      if (t + 1 < in.ntiles) produce_and_publish(t + 1, t + 1, Pass1Layout{});
      consume(T / 2, T);
      // this warp is done with buffer b
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bars[4 + b])) : "memory");
      if (b) ccnt1++;
      else ccnt0++;
      // tile merge: best (doubled) with tie bit, and first tile reaching it
      const uint32_t tpk = (uint32_t)t * 0x10001u;
#pragma unroll
      for (int v = 0; v < P; v++) {
        const uint32_t mb = m1[v] & 0xFFFEFFFEu;
        const uint32_t gt = __vcmpgtu2(tmax[v], m1[v]);
        const uint32_t eq = __vcmpeq2(tmax[v], mb);
        if (GAP) {
          // the tile that is not (or no longer) the first best one joins the other tiles' maximum
          uint32_t* m2 = st_best + v * kThreads + tid;
          *m2 = vmax2(*m2, (gt & mb) | (~gt & tmax[v]));
        }
        m1[v] = (gt & tmax[v]) | (~gt & (m1[v] | (eq & 0x00010001u)));
        ts[v] = (gt & tpk) | (~gt & ts[v]);
        tmax[v] = 0u;
      }
    }
    __syncthreads();  // pass 2 re-stages the buffers: every warp is done with them
    if (s_abort) break;

    // ================= classify: a field stays a candidate (best >= 2) only if its
    // minimum was reached in a single tile (or labels are wanted); others resolve to -1
    // (cmask: bit 2v + h marks a candidate, which pass 2 resolves)
    unsigned long long cmask = 0;  // 2P <= 64 fields
#pragma unroll
    for (int v = 0; v < P; v++) {
      uint32_t mv = m1[v], tv = ts[v];
      const uint32_t m2v = GAP ? st_best[v * kThreads + tid] : 0u;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        if (GAP) {
          // another tile within T of the best: the best is not unique (marked like a tie)
          const uint32_t f2 = (m2v >> (16 * h)) & 0xFFFFu;
          if (f2 != 0u && ((mv >> (16 * h)) & 0xFFFEu) < f2 + p.gap2) mv |= 1u << (16 * h);
        }
        const uint32_t field = (mv >> (16 * h)) & 0xFFFFu;
        const uint32_t rw = (uint32_t)h | ((uint32_t)v << 1) | role_hi;
        const bool valid = nroles >= K::ROLES || (rw >> nroles) == 0u;
        const bool cand = valid && field > 1u && (want_aux || !(field & 1u));
        if (!cand) {
          mv &= ~(0xFFFFu << (16 * h));
          tv |= 0xFFFFu << (16 * h);
        } else {
          cmask |= 1ull << (2 * v + h);
        }
      }
      st_best[v * kThreads + tid] = mv;
      st_tile[v * kThreads + tid] = tv;
    }

    // ================= pass-2 work list: the CTA's candidates grouped by their best tile, one
    // 16-bit entry (thread << 6 | field) each, in this CTA's global scratch; counted and placed with
    // shared-memory atomics in the idle coefficient area.  Every warp then takes a share of each
    // tile's candidates, whoever owns them, so no warp holds up the others with a long list.
    uint16_t* wl = p.wlist + (size_t)blockIdx.x * p.wl_stride;
    uint16_t* woff = wl + (1u << kRoles);      // ntiles + 1 offsets
    uint16_t* wtiles = woff + in.ntiles + 1;  // the tiles that hold candidates, ascending; then their count
    unsigned* whist = coefbuf;
    for (int i = tid; i <= in.ntiles; i += kThreads) whist[i] = 0u;
    __syncthreads();
    for (unsigned long long m = cmask; m; m &= m - 1) {
      const int c = __ffsll((long long)m) - 1;
      atomicAdd(&whist[(st_tile[(c >> 1) * kThreads + tid] >> (16 * (c & 1))) & 0xFFFFu], 1u);
    }
    __syncthreads();
    if (warp == 0) {
      // exclusive scan of the tile counts: each lane sums a run of tiles, then a warp scan
      const int per = (in.ntiles + 32) / 32;
      const int i0 = lane * per, i1 = min(i0 + per, in.ntiles + 1);
      unsigned run = 0;
      for (int i = i0; i < i1; i++) run += whist[i];
      unsigned incl = run;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += y;
      }
      unsigned at = incl - run, nonempty = 0;
      for (int i = i0; i < i1; i++) {
        const unsigned c = whist[i];
        woff[i] = (uint16_t)at;
        whist[i] = at;  // becomes the placement cursor
        at += c;
        nonempty += (i < in.ntiles && c != 0u) ? 1u : 0u;
      }
      __syncwarp();  // whist now holds the offsets: tile i has whist[i + 1] - whist[i] candidates
      // the tiles that hold candidates, ascending, and their number at wtiles[ntiles]
      unsigned nincl = nonempty;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, nincl, d);
        if (lane >= d) nincl += y;
      }
      unsigned w = nincl - nonempty;
      for (int i = i0; i < min(i1, in.ntiles); i++)
        if (whist[i + 1] != whist[i]) wtiles[w++] = (uint16_t)i;
      if (lane == 31) wtiles[in.ntiles] = (uint16_t)nincl;
    }
    __syncthreads();
    for (unsigned long long m = cmask; m; m &= m - 1) {
      const int c = __ffsll((long long)m) - 1;
      const unsigned t = (st_tile[(c >> 1) * kThreads + tid] >> (16 * (c & 1))) & 0xFFFFu;
      wl[atomicAdd(&whist[t], 1u)] = (uint16_t)((tid << 6) | c);
    }
    __syncthreads();  // the list and offsets are visible to the CTA; the coefficient area is free again
    // st_best / st_tile as 16-bit fields: field (v, h) of thread x is halfword 2 (v THREADS + x) + h
    uint16_t* best16 = reinterpret_cast<uint16_t*>(st_best);
    uint16_t* tile16 = reinterpret_cast<uint16_t*>(st_tile);

    // ================= pass 2: re-stage each tile and resolve its candidates.  The records of
    // tile t + 1 are produced (pass-2 layout) before tile t is resolved, with the hand-over of pass 1
    // (produced / consumed mbarriers).
    // only the tiles that hold candidates are staged and produced again
    const int n2 = wtiles[in.ntiles];
    if (n2 > 0) {
      prefetch_first_tiles<T>(in, rawbuf, bars, issued, wtiles[0], n2 > 1 ? (int)wtiles[1] : -1);
      produce_and_publish(0, wtiles[0], Pass2Layout{});
    }
    for (int i2 = 0; i2 < n2; i2++) {
      const int b = i2 & 1;
      const int t = wtiles[i2];
      if (!mbar_wait(&bars[2 + b], (b ? fcnt1 : fcnt0) & 1u, p.spin_handover)) {
        atomicOr(p.ctrl, kErrTimeout);
        s_abort = 1;
      }
      if (b) fcnt1++;
      else fcnt0++;
      if (s_abort) break;
      // every producer has read raw[b] (the i2-th listed tile): refill it with the (i2 + 2)-th
      if (i2 + 2 < n2) {
        if (tid == 0)
          bulk_load(rawbuf + b * T * in.rec_words, in.rec + (size_t)wtiles[i2 + 2] * T * in.rec_words,
                    (unsigned)(T * in.rec_words * 4), &bars[b]);
        issued[b]++;
      }
      if (i2 + 1 < n2) produce_and_publish(i2 + 1, wtiles[i2 + 1], Pass2Layout{});
      const uint32_t* cbuf = coefbuf + b * T * K::CS2;
      const int e0 = woff[t], e1 = woff[t + 1];
      // a tile with at least 32 candidates per warp: each lane scores one candidate against every
      // conformation of the tile (no votes, independent steps); the rest one candidate per warp
      const int nlane = (e1 - e0) / (32 * K::NW) * (32 * K::NW);
      for (int base = e0 + 32 * warp; base < e0 + nlane; base += 32 * K::NW) {
        const uint32_t ent = wl[base + lane];
        const int owner = (int)(ent >> 6), c = (int)(ent & 63u), v = c >> 1, h = c & 1;
        const int src = owner & 31, wo = owner >> 5;
        const int fi = 2 * (v * kThreads + owner) + h;
        const uint32_t sfld = best16[fi];
        const uint32_t want = sfld & 0xFFFEu;
        int count = 0, first = 0x7FFFFFFF;
#pragma unroll 4
        for (int sc = 0; sc < T; sc++) {
          const uint32_t* cs = cbuf + sc * K::CS2;
          uint32_t x = cs[src] + cs[K::WT_OFF + wo];
#pragma unroll
          for (int j = 0; j < R - 1; j++) x += ((v >> j) & 1) ? cs[K::TP_OFF + j] : 0u;
          const uint32_t xf = (x >> (16 * h)) & 0xFFFFu;
          if (xf == want) {  // padding scores 0 never match
            first = min(first, sc);
            if (!GAP) count++;
          }
          if (GAP && xf >= 2u && xf + p.gap2 > want) count++;
        }
        const bool unique = !(sfld & 1u) && count == 1;
        best16[fi] = first != 0x7FFFFFFF ? (uint16_t)(((uint32_t)first << 1) | (unique ? 1u : 0u)) : (uint16_t)0;
        if (first == 0x7FFFFFFF) tile16[fi] = 0xFFFFu;
      }
      for (int e = e0 + nlane + warp; e < e1; e += K::NW) {
        const uint32_t ent = wl[e];
        const int owner = (int)(ent >> 6), c = (int)(ent & 63u), v = c >> 1, h = c & 1;
        const int src = owner & 31, wo = owner >> 5;
        const int fi = 2 * (v * kThreads + owner) + h;
        const uint32_t sfld = best16[fi];
        const uint32_t want = sfld & 0xFFFEu;
        // lane l checks conformations l, l + 32, ... of the tile; the steps are independent
        int count = 0, first = 0x7FFFFFFF;
#pragma unroll
        for (int i = 0; i < T; i += 32) {
          const uint32_t* cs = cbuf + (i + lane) * K::CS2;
          uint32_t x = cs[src] + cs[K::WT_OFF + wo];
#pragma unroll
          for (int j = 0; j < R - 1; j++)
            if ((v >> j) & 1) x += cs[K::TP_OFF + j];
          const uint32_t xf = (x >> (16 * h)) & 0xFFFFu;
          const uint32_t bal = __ballot_sync(0xFFFFFFFFu, xf == want);  // padding scores 0 never match
          if (bal) first = min(first, i + __ffs(bal) - 1);
          if (GAP)  // real conformations (padding is 0) within T of the best, the best included
            count += __popc(__ballot_sync(0xFFFFFFFFu, xf >= 2u && xf + p.gap2 > want));
          else
            count += __popc(bal);
        }
        if (lane == 0) {
          // (index in the tile << 1 | unique) beside the tile; the class is looked up after pass 2,
          // when the loads of all fields can be in flight together
          const bool unique = !(sfld & 1u) && count == 1;
          best16[fi] = first != 0x7FFFFFFF ? (uint16_t)(((uint32_t)first << 1) | (unique ? 1u : 0u)) : (uint16_t)0;
          if (first == 0x7FFFFFFF) tile16[fi] = 0xFFFFu;
        }
      }
      // this warp is done with buffer b
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bars[4 + b])) : "memory");
      if (b) ccnt1++;
      else ccnt0++;
    }
    __syncthreads();  // every warp is done with the buffers (the next item's pass 1 refills them)
    if (s_abort) break;
    // class ids of this thread's fields: (tile, index in the tile) -> conformation -> class, into
    // the final encoding (st_tile: class or 0xFFFF for none; st_best: 1 where the minimum is unique)
#pragma unroll 4
    for (int v = 0; v < P; v++) {
      const uint32_t mv = st_best[v * kThreads + tid], tv = st_tile[v * kThreads + tid];
      uint32_t nb = 0u, nt = 0u;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const uint32_t tf = (tv >> (16 * h)) & 0xFFFFu, bf = (mv >> (16 * h)) & 0xFFFFu;
        const uint32_t cls = tf == 0xFFFFu ? 0xFFFFu : (uint32_t)in.conf_class[tf * T + (bf >> 1)] & 0xFFFFu;
        nt |= cls << (16 * h);
        nb |= (bf & 1u) << (16 * h);
      }
      st_best[v * kThreads + tid] = nb;
      st_tile[v * kThreads + tid] = nt;
    }

    // reversal mirror of this item's ids (only for non-palindromic odd patterns); when every free
    // even residue is a role of this CTA, the mirrored ids are written in a second, coalesced pass
    // (computed here, not at the top of the item, so that nothing extra stays live through pass 1)
    const uint32_t o_rev = bd.otab ? (__brev(o) >> (32 - bd.no_free)) : o;  // no_free >= 1 with a table
    const bool mirror = bd.otab != nullptr && o_rev != o;
    const bool mirror_gather = mirror && bd.ne_free == bd.nroles;

    // ================= write the two sequences of each packed register (ids differ in bit 0)
    for (int v = 0; v < P; v++) {
      const uint32_t mv = st_best[v * kThreads + tid], tv = st_tile[v * kThreads + tid];
      int ph[2], ax[2];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const uint32_t tf = (tv >> (16 * h)) & 0xFFFFu;
        ax[h] = tf == 0xFFFFu ? -1 : (int)tf;
        ph[h] = ((mv >> (16 * h)) & 0xFFFFu) == 1u ? ax[h] : -1;
      }
      const uint32_t rw0 = ((uint32_t)v << 1) | role_hi;
      const bool valid0 = nroles >= K::ROLES || (rw0 >> nroles) == 0u;
      const bool valid1 = nroles >= K::ROLES || ((rw0 | 1u) >> nroles) == 0u;
      if (!valid0) continue;
      const uint32_t e0 = (rw0 & role_mask) | ehigh;
      const unsigned long long g0 = interleave(e0, o);
      const unsigned long long idx = bd.out_off + (g0 - bd.g_base);
      int32_t* ph_out = in.phen;
      int32_t* ax_out = in.aux;
      if (mirror && !mirror_gather) {
        // P(h^R) = P(h) and the lowest minimising class is the same: write the reversed ids too
        const uint32_t nbits_e = bd.ne_free;
        const unsigned long long gm0 = interleave(__brev(e0) >> (32 - nbits_e), o_rev);
        ph_out[bd.out_off + (gm0 - bd.g_base)] = ph[0];
        if (want_aux) ax_out[bd.out_off + (gm0 - bd.g_base)] = ax[0];
        if (valid1) {
          const unsigned long long gm1 = interleave(__brev(e0 | 1u) >> (32 - nbits_e), o_rev);
          ph_out[bd.out_off + (gm1 - bd.g_base)] = ph[1];
          if (want_aux) ax_out[bd.out_off + (gm1 - bd.g_base)] = ax[1];
        }
      }
      const bool pair_ok = valid1 && ((reinterpret_cast<uintptr_t>(ph_out + idx) & 7u) == 0u) &&
                           (!want_aux || (reinterpret_cast<uintptr_t>(ax_out + idx) & 7u) == 0u);
      if (pair_ok) {
        *reinterpret_cast<int2*>(ph_out + idx) = make_int2(ph[0], ph[1]);
        if (want_aux) *reinterpret_cast<int2*>(ax_out + idx) = make_int2(ax[0], ax[1]);
      } else {
        ph_out[idx] = ph[0];
        if (want_aux) ax_out[idx] = ax[0];
        if (valid1) {
          ph_out[idx + 1] = ph[1];
          if (want_aux) ax_out[idx + 1] = ax[1];
        }
      }
    }
    if (mirror_gather) {
      // write id (rev(e), rev(o)) for this thread's own role pattern e; its result is the one of
      // (rev(e), o) = roles of another thread, read from the shared-memory state
      __syncthreads();
      const int nbits_e = (int)bd.ne_free;
      for (int v = 0; v < P; v++) {
        int ph[2], ax[2];
        const uint32_t rw0 = ((uint32_t)v << 1) | role_hi;
        const bool valid0 = nroles >= K::ROLES || (rw0 >> nroles) == 0u;
        const bool valid1 = nroles >= K::ROLES || ((rw0 | 1u) >> nroles) == 0u;
        if (!valid0) continue;
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const uint32_t src = __brev((rw0 | (uint32_t)h) & role_mask) >> (32 - nbits_e);  // roles of the source id
          const uint32_t sh = src & 1u, sv = (src >> 1) & (uint32_t)(P - 1);
          const uint32_t stid = ((src >> R) & 31u) + 32u * (src >> (R + kLaneRoles));
          const uint32_t mv = st_best[sv * kThreads + stid], tv = st_tile[sv * kThreads + stid];
          const uint32_t tf = (tv >> (16 * sh)) & 0xFFFFu;
          ax[h] = tf == 0xFFFFu ? -1 : (int)tf;
          ph[h] = ((mv >> (16 * sh)) & 0xFFFFu) == 1u ? ax[h] : -1;
        }
        const unsigned long long g0 = interleave(rw0 & role_mask, o_rev);
        const unsigned long long idx = bd.out_off + (g0 - bd.g_base);
        int32_t* ph_out = in.phen;
        int32_t* ax_out = in.aux;
        const bool pair_ok = valid1 && ((reinterpret_cast<uintptr_t>(ph_out + idx) & 7u) == 0u) &&
                             (!want_aux || (reinterpret_cast<uintptr_t>(ax_out + idx) & 7u) == 0u);
        if (pair_ok) {
          *reinterpret_cast<int2*>(ph_out + idx) = make_int2(ph[0], ph[1]);
          if (want_aux) *reinterpret_cast<int2*>(ax_out + idx) = make_int2(ax[0], ax[1]);
        } else {
          ph_out[idx] = ph[0];
          if (want_aux) ax_out[idx] = ax[0];
          if (valid1) {
            ph_out[idx + 1] = ph[1];
            if (want_aux) ax_out[idx + 1] = ax[1];
          }
        }
      }
    }
    // the state area and s_item are rewritten by the next item (barriers at its top)
  }
  // after an abort, wait (with the fixed bound) for bulk copies still in flight before exiting; a
  // copy that does not land in time may still write into shared memory that a later CTA owns, so
  // that is reported as its own error and the host treats the whole launch as invalid
  if (tid == 0) {
    for (int k = 0; k < 2; k++)
      while (waited[k] < issued[k]) {
        if (!mbar_wait(&bars[k], waited[k] & 1u, kSpinLimit)) {
          atomicOr(p.ctrl, kErrDrain);
          break;
        }
        waited[k]++;
      }
  }
}

template <class K>
size_t smem_bytes(int max_rec_words) {
  const size_t words = (size_t)K::kCoefWords + 2ull * K::T * max_rec_words + (size_t)K::kStateWords;
  return words * 4 + 6 * sizeof(uint64_t);
}

// Grid of a launch of this shape (one wave of resident CTAs, at most one per work item), and with
// `launch` set the launch itself.
template <class K, bool GAP = false>
int shape_grid_or_launch(const hp::PhenParams& prm, cudaStream_t stream, unsigned grid_limit, unsigned* grid_out,
                         bool launch) {
  const size_t smem = smem_bytes<K>(prm.max_rec_words);
  auto kern = phenotype_kernel<K, GAP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return hp::cuda_fail(e, "cudaFuncSetAttribute(phenotype_kernel)");
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K::THREADS, smem);
  if (e != cudaSuccess) return hp::cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (per_sm < 1) return hp::fail(HP_EUNSUPPORTED, "phenotype kernel shape does not fit on this GPU");
  unsigned long long grid = (unsigned long long)sms * per_sm;
  if (grid > prm.total_items) grid = prm.total_items;
  if (grid_limit && grid > grid_limit) grid = grid_limit;
  if (grid < 1) grid = 1;
  if (grid_out) *grid_out = (unsigned)grid;
  if (!launch) return HP_OK;
  if (!prm.wlist || prm.wl_ctas < grid) return hp::fail(HP_EINVAL, "phenotype kernel: work lists not set up for the grid");
  kern<<<(unsigned)grid, K::THREADS, smem, stream>>>(prm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return hp::cuda_fail(e, "phenotype_kernel launch");
  return HP_OK;
}

}  // namespace

namespace hp {

void small_roles_shape(int max_ne_free, int* roles, int* reg_bits, int* tile) {
  *roles = max_ne_free >= kRoles ? kRoles : std::max(max_ne_free, 11);
  if (*roles == 13 || *roles == 12) {
    *reg_bits = 5;
    *tile = 128;
  } else if (*roles == 11) {
    *reg_bits = 4;
    *tile = 64;
  }
}

bool tile_cfg_supported(int reg_bits, int tile) {
  switch (reg_bits * 1000 + tile) {
    case 4064: case 4128: case 5064: case 5128: case 5256: case 6064: case 6128: case 6256:
      return true;
    default:
      return false;
  }
}

void default_tile_cfg(int* reg_bits, int* tile) {
  *reg_bits = 5;
  *tile = 256;
}

namespace {
int grid_or_launch(const PhenParams& prm, int reg_bits, int tile, cudaStream_t stream, unsigned grid_limit,
                   unsigned* grid, bool launch) {
  // thresholds above 1 have one compiled shape (the default)
  if (prm.gap2 > 2u) return shape_grid_or_launch<Cfg<5, 256>, true>(prm, stream, grid_limit, grid, launch);
  // fewer roles per CTA: one compiled shape each (small_roles_shape)
  switch (prm.roles) {
    case 13: return shape_grid_or_launch<Cfg<5, 128, 13>>(prm, stream, grid_limit, grid, launch);
    case 12: return shape_grid_or_launch<Cfg<5, 128, 12>>(prm, stream, grid_limit, grid, launch);
    case 11: return shape_grid_or_launch<Cfg<4, 64, 11>>(prm, stream, grid_limit, grid, launch);
    case kRoles: break;
    default: return fail(HP_EINVAL, "unsupported role count");
  }
  switch (reg_bits * 1000 + tile) {
    case 4064: return shape_grid_or_launch<Cfg<4, 64>>(prm, stream, grid_limit, grid, launch);
    case 4128: return shape_grid_or_launch<Cfg<4, 128>>(prm, stream, grid_limit, grid, launch);
    case 5064: return shape_grid_or_launch<Cfg<5, 64>>(prm, stream, grid_limit, grid, launch);
    case 5128: return shape_grid_or_launch<Cfg<5, 128>>(prm, stream, grid_limit, grid, launch);
    case 5256: return shape_grid_or_launch<Cfg<5, 256>>(prm, stream, grid_limit, grid, launch);
    case 6064: return shape_grid_or_launch<Cfg<6, 64>>(prm, stream, grid_limit, grid, launch);
    case 6128: return shape_grid_or_launch<Cfg<6, 128>>(prm, stream, grid_limit, grid, launch);
    case 6256: return shape_grid_or_launch<Cfg<6, 256>>(prm, stream, grid_limit, grid, launch);
    default: return fail(HP_EINVAL, "unsupported tile configuration");
  }
}
}  // namespace

int launch_phenotype(const PhenParams& prm, int reg_bits, int tile, cudaStream_t stream, unsigned grid_limit) {
  return grid_or_launch(prm, reg_bits, tile, stream, grid_limit, nullptr, true);
}

int launch_block_bytes(const PhenParams& prm, int reg_bits, int tile, unsigned grid_limit, size_t* bytes,
                       unsigned* ctas) {
  unsigned grid = 0;
  const int rc = grid_or_launch(prm, reg_bits, tile, nullptr, grid_limit, &grid, false);
  if (rc != HP_OK) return rc;
  int max_tiles = 0;
  for (int i = 0; i < prm.ninst; i++) max_tiles = std::max(max_tiles, prm.inst[i].ntiles);
  // uint16: 2^14 entries, ntiles + 1 offsets, ntiles + 1 listed tiles and their count; 128-byte rows
  const size_t stride = ((size_t)(1u << kRoles) + 2 * ((size_t)max_tiles + 1) + 63) / 64 * 64;
  *ctas = grid;
  *bytes = 256 + stride * 2 * grid;
  return HP_OK;
}

void bind_launch_block(PhenParams& prm, void* block, unsigned ctas) {
  int max_tiles = 0;
  for (int i = 0; i < prm.ninst; i++) max_tiles = std::max(max_tiles, prm.inst[i].ntiles);
  prm.ctrl = static_cast<unsigned*>(block);
  prm.wlist = reinterpret_cast<uint16_t*>(static_cast<char*>(block) + 256);
  prm.wl_stride = (unsigned)(((size_t)(1u << kRoles) + 2 * ((size_t)max_tiles + 1) + 63) / 64 * 64);
  prm.wl_ctas = ctas;
}

bool half_enumeration_enabled() {
  static const bool on = [] {
    const char* e = getenv("HP_FULL_ENUMERATION");
    return !(e && e[0] == '1');
  }();
  return on;
}

int half_tables(const hp_structs* cs, DevTables** out) {
  DevTables* dt = nullptr;
  int rc = device_tables(cs, &dt);
  if (rc != HP_OK) return rc;
  hp_structs* s = const_cast<hp_structs*>(cs);
  std::lock_guard<std::mutex> lock(s->mu);
  if (!dt->half_otab) {
    const int no = s->NO;
    std::vector<uint32_t> tab;
    for (uint32_t o = 0; o < (1u << no); o++) {
      uint32_t r = 0;
      for (int j = 0; j < no; j++) r |= ((o >> j) & 1u) << (no - 1 - j);
      if (o <= r) tab.push_back(o);
    }
    cudaError_t e = cudaMalloc(&dt->half_otab, tab.size() * 4);
    if (e == cudaSuccess) e = cudaMemcpy(dt->half_otab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(dt->half_otab);
      dt->half_otab = nullptr;
      return cuda_fail(e, "reversal tables");
    }
    dt->half_n = (int)tab.size();
  }
  *out = dt;
  return HP_OK;
}

int plan_phenotype(const hp_structs* const* libs, const uint64_t* begins, const uint64_t* counts, int n,
                   int32_t* const* d_phen, int32_t* const* d_aux, int tile, PhenParams& prm, int roles) {
  if (roles != kRoles && roles != 13 && roles != 12 && roles != 11) return fail(HP_EINVAL, "unsupported role count");
  prm.roles = roles;
  if (n < 1 || n > kPhenMaxInst)
    return fail(HP_EINVAL, "a batch holds 1 to " + std::to_string(kPhenMaxInst) + " instances");
  // instances with more conformations first, so the dynamic queue ends on cheap items
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  for (int i = 0; i < n; i++)
    if (!libs[i] || !d_phen || !d_phen[i]) return fail(HP_EINVAL, "batch entry " + std::to_string(i) + ": NULL library or output");
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return libs[a]->S_dir > libs[b]->S_dir; });
  prm.ninst = n;
  prm.max_rec_words = 0;
  prm.one = 1u;
  prm.gap2 = 2u;
  prm.spin = wait_limit(kSpinLimit);
  prm.spin_handover = wait_limit(1ll << 22);
  unsigned long long items = 0;
  int nb = 0;
  for (int q = 0; q < n; q++) {
    const int i = order[q];
    const hp_structs* s = libs[i];
    if (s->N > 2 * kMaxHalf) return fail(HP_EUNSUPPORTED, "N > 40");
    if (s->S >= 0xFFFF) return fail(HP_EUNSUPPORTED, "more than 65534 classes");
    const unsigned long long space = 1ull << s->N;
    if (begins[i] >= space || counts[i] > space - begins[i])
      return fail(HP_EINVAL, "batch entry " + std::to_string(i) + ": sequence range exceeds 2^N");
    DevTables* dt = nullptr;
    int rc = device_tables(s, &dt);
    if (rc != HP_OK) return rc;
    PhenInst& in = prm.inst[q];
    in.rec = dt->rec;
    in.conf_class = dt->conf_class;
    in.phen = d_phen[i];
    in.aux = d_aux ? d_aux[i] : nullptr;
    in.S_dir = s->S_dir;
    in.ntiles = (s->S_dir + tile - 1) / tile;
    in.rec_words = s->rec_words;
    in.NE = s->NE;
    prm.max_rec_words = std::max(prm.max_rec_words, s->rec_words);
    // aligned power-of-two blocks of [begin, begin + count)
    unsigned long long pos = begins[i], end = begins[i] + counts[i];
    while (pos < end) {
      int m = 0;
      while (m < 63) {
        const unsigned long long size = 1ull << (m + 1);
        if ((pos & (size - 1)) != 0 || pos + size > end) break;
        m++;
      }
      if (nb >= kPhenMaxBlocks) return fail(HP_EUNSUPPORTED, "sequence ranges split into too many aligned blocks");
      PhenBlock& d = prm.blocks[nb++];
      d.g_base = pos;
      d.out_off = pos - begins[i];
      d.item_begin = items;
      d.ne_free = (unsigned)std::min((m + 1) / 2, s->NE);
      d.no_free = (unsigned)std::min(m / 2, s->NO);
      d.nroles = (unsigned)std::min((int)d.ne_free, roles);
      d.inst = (unsigned)q;
      d.otab = nullptr;
      d.ntab = 0;
      d.pad = 0;
      if (m == s->N && (s->N & 1) && s->NO >= 1 && half_enumeration_enabled()) {
        // the whole space of an odd-length chain: compute one id of every reversal pair
        DevTables* ht = nullptr;
        rc = half_tables(s, &ht);
        if (rc != HP_OK) return rc;
        d.otab = ht->half_otab;
        d.ntab = (unsigned)ht->half_n;
        items += (unsigned long long)d.ntab << (d.ne_free - d.nroles);
      } else {
        items += (1ull << d.no_free) << (d.ne_free - d.nroles);
      }
      pos += 1ull << m;
    }
  }
  prm.nblocks = nb;
  prm.total_items = items;
  return HP_OK;
}

int role_classes(const hp_structs* const* libs, const uint64_t* begins, const uint64_t* counts, int n,
                 int32_t* const* d_phen, int tile, std::vector<int>& cls) {
  PhenParams* tmp = new (std::nothrow) PhenParams();
  if (!tmp) return fail(HP_ENOMEM, "out of host memory");
  cls.assign(n, kRoles);
  for (int i = 0; i < n; i++) {
    const int rc = plan_phenotype(&libs[i], &begins[i], &counts[i], 1, &d_phen[i], nullptr, tile, *tmp);
    if (rc != HP_OK) {
      delete tmp;
      return rc;
    }
    int max_ne = 0, r = 0, t = 0;
    for (int k = 0; k < tmp->nblocks; k++) max_ne = std::max(max_ne, (int)tmp->blocks[k].ne_free);
    small_roles_shape(max_ne, &cls[i], &r, &t);
  }
  delete tmp;
  return HP_OK;
}

int run_phenotype(const hp_structs* const* libs, const uint64_t* begins, const uint64_t* counts, int n,
                  int32_t* const* d_phen, int32_t* const* d_aux, int reg_bits, int tile, cudaStream_t st,
                  unsigned grid_limit, int gap_threshold, bool auto_roles) {
  if (!tile_cfg_supported(reg_bits, tile)) return fail(HP_EINVAL, "unsupported tile configuration");
  if (gap_threshold < 1 || gap_threshold > (1 << 20)) return fail(HP_EINVAL, "gap_threshold must be in [1, 2^20]");
  if (gap_threshold > 1) {
    reg_bits = 5;  // the shape compiled for thresholds above 1
    tile = 256;
    auto_roles = false;
  }
  if (auto_roles && n > 1) {
    // boxes that need different role counts: one persistent launch per role count, each over all the
    // boxes of that count, back to back on the stream
    std::vector<int> cls;
    int rc = role_classes(libs, begins, counts, n, d_phen, tile, cls);
    if (rc != HP_OK) return rc;
    if (std::any_of(cls.begin(), cls.end(), [&](int c) { return c != cls[0]; })) {
      for (const int c : {kRoles, 13, 12, 11}) {
        std::vector<const hp_structs*> l;
        std::vector<uint64_t> b, k;
        std::vector<int32_t*> o, a;
        for (int i = 0; i < n; i++)
          if (cls[i] == c) {
            l.push_back(libs[i]);
            b.push_back(begins[i]);
            k.push_back(counts[i]);
            o.push_back(d_phen[i]);
            a.push_back(d_aux ? d_aux[i] : nullptr);
          }
        if (l.empty()) continue;
        rc = run_phenotype(l.data(), b.data(), k.data(), (int)l.size(), o.data(), d_aux ? a.data() : nullptr, reg_bits,
                           tile, st, grid_limit, gap_threshold, true);
        if (rc != HP_OK) return rc;
      }
      return HP_OK;
    }
  }
  PhenParams* prm = new (std::nothrow) PhenParams();
  if (!prm) return fail(HP_ENOMEM, "out of host memory");
  int rc = plan_phenotype(libs, begins, counts, n, d_phen, d_aux, tile, *prm);
  if (rc == HP_OK && auto_roles) {
    // every block has fewer than 14 free even residues (a small box or a short range): a shape with
    // as many roles per CTA as there are, so that no CTA evaluates patterns it then drops
    int max_ne = 0;
    for (int i = 0; i < prm->nblocks; i++) max_ne = std::max(max_ne, (int)prm->blocks[i].ne_free);
    int roles = kRoles;
    small_roles_shape(max_ne, &roles, &reg_bits, &tile);
    if (roles != kRoles) rc = plan_phenotype(libs, begins, counts, n, d_phen, d_aux, tile, *prm, roles);
  }
  prm->gap2 = 2u * (uint32_t)gap_threshold;
  if (rc != HP_OK || prm->total_items == 0) {
    delete prm;
    return rc;
  }
  size_t bytes = 0;
  unsigned ctas = 0;
  rc = launch_block_bytes(*prm, reg_bits, tile, grid_limit, &bytes, &ctas);
  if (rc != HP_OK) {
    delete prm;
    return rc;
  }
  void* block = nullptr;
  cudaError_t e = cudaMallocAsync(&block, bytes, st);
  if (e != cudaSuccess) {
    delete prm;
    return cuda_fail(e, "cudaMallocAsync(phenotype control words and work lists)");
  }
  unsigned* ctrl = static_cast<unsigned*>(block);
  cudaMemsetAsync(ctrl, 0, kPhenCtrlBytes, st);
  bind_launch_block(*prm, block, ctas);
  rc = launch_phenotype(*prm, reg_bits, tile, st, grid_limit);
  delete prm;
  unsigned herr = 0;
  if (rc == HP_OK) {
    e = cudaMemcpyAsync(&herr, ctrl, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "phenotype kernel execution");
  }
  cudaFreeAsync(ctrl, st);
  if (rc == HP_OK && (herr & kErrDrain))
    rc = fail(HP_ETIMEOUT, "phenotype kernel: a wait timed out and bulk copies were still in flight at exit; "
                           "the output is invalid");
  else if (rc == HP_OK && (herr & kErrTimeout))
    rc = fail(HP_ETIMEOUT, "phenotype kernel: a bounded wait timed out; the output is invalid");
  return rc;
}

}  // namespace hp

extern "C" int hp_phenotype_map(const hp_structs* s, uint64_t seq_begin, uint64_t seq_count, int32_t gap_threshold,
                                int32_t* d_phen, int32_t* d_argmin_aux, void* stream) {
  if (!s) return hp::fail(HP_EINVAL, "hp_phenotype_map: library is NULL");
  if (!d_phen) return hp::fail(HP_EINVAL, "hp_phenotype_map: d_phen is NULL");
  if (gap_threshold < 1 || gap_threshold > (1 << 20))
    return hp::fail(HP_EINVAL, "hp_phenotype_map: gap_threshold must be in [1, 2^20]");
  if (s->N > 2 * hp::kMaxHalf) return hp::fail(HP_EUNSUPPORTED, "hp_phenotype_map: N > 40");
  if (seq_count == 0) return HP_OK;
  const unsigned long long space = 1ull << s->N;
  if (seq_begin >= space || seq_count > space - seq_begin)
    return hp::fail(HP_EINVAL, "hp_phenotype_map: sequence range exceeds 2^N");
  int r = s->tile_reg_bits, t = s->tile_size;
  const bool auto_roles = r == 0;  // no shape set on the library: pick the role count from the range
  if (!r) hp::default_tile_cfg(&r, &t);
  return hp::run_phenotype(&s, &seq_begin, &seq_count, 1, &d_phen, d_argmin_aux ? &d_argmin_aux : nullptr, r, t,
                           (cudaStream_t)stream, 0, gap_threshold, auto_roles);
}
