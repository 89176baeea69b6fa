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
// Layout of the even-pattern bits ("roles"), R = register bits (template):
//   role 0          split: low/high 16-bit half of a packed register
//   roles 1..R-1    tree: index of one of the 2^(R-1) packed registers
//   roles R..R+4    lane of the warp
//   roles R+5..R+7  warp of the CTA (8 warps)
// Each thread keeps, per packed register, the running maximum of the doubled,
// biased score 2 (x + 1) of two sequences (max.u16x2).  Per tile of T
// conformations the tile maximum is merged into a best value with a tie bit
// and the tile index where the best was first reached.  A sequence whose best
// is reached in two tiles is not unique; the others re-scan that one tile in
// the epilogue (a warp-cooperative exact count with ballots), which also finds
// the lowest-index conformation at the minimum.
//
// Data movement.  Conformation records (contact masks, see hp_internal.h) are
// staged tile by tile into shared memory with the bulk-copy engine
// (cp.async.bulk + mbarrier, bounded waits), double buffered; one thread per
// conformation turns a record into the CTA's coefficient record (lane table,
// warp table, packed tree coefficients) in a second double buffer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "hp_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kLaneRoles = 5;
constexpr int kWarpRoles = 3;
constexpr int kCStride = 52;      // words per coefficient record (13 x 16 B, odd in 16-B units)
constexpr int kMaxBlocks = 96;    // aligned id blocks per launch
constexpr unsigned kErrTimeout = 1u;
constexpr long long kSpinLimit = 1ll << 26;

struct BlockDesc {
  unsigned long long g_base;      // first sequence id of the block (aligned to 2^m)
  unsigned long long out_off;     // index of g_base in the output
  unsigned long long item_begin;  // first work item of the block
  unsigned int ne_free, no_free;  // even / odd residues below bit m
  unsigned int nroles;            // real roles: min(ne_free, R + 8)
  unsigned int pad;
};

struct Params {
  const uint32_t* rec;  // conformation records, padded to a multiple of T
  const int32_t* conf_class;
  int32_t* phen;
  int32_t* aux;
  unsigned int* err;
  int S_dir, ntiles, rec_words, NE, NO;
  int nblocks;
  unsigned long long total_items;
  BlockDesc blocks[kMaxBlocks];
};

__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Wait for phase `parity` of the barrier; false after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (long long i = 0; i < kSpinLimit; i++) {
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
__device__ __forceinline__ uint32_t coef(uint32_t mask, uint32_t o) {
  return 10u * __popc(mask) + 3u * __popc(mask & o);
}
// score part that depends on the odd residues only: 10 sum_j o_j c_j
__device__ __forceinline__ uint32_t odd_part(const uint32_t* r, int NE, uint32_t o) {
  return 10u * (__popc(o & r[NE]) + 2u * __popc(o & r[NE + 1]) + 4u * __popc(o & r[NE + 2]));
}

template <int R, int T>
struct Smem {
  static constexpr int P = 1 << (R - 1);
  static constexpr int kCoefWords = 2 * T * kCStride;
  static constexpr int kStateWords = 2 * P * kThreads;
};

template <int R, int T>
__global__ void __launch_bounds__(kThreads, 1) phenotype_kernel(const __grid_constant__ Params p) {
  constexpr int P = 1 << (R - 1);
  constexpr int NROLE = R + kLaneRoles + kWarpRoles;
  extern __shared__ __align__(128) uint32_t smem[];
  // layout: [coef 2 x T x kCStride][raw 2 x T x rec_words] ... [2 mbarriers]; the
  // epilogue reuses the front as per-thread state (2 x P x kThreads words)
  uint32_t* coefbuf = smem;
  const int coef_words = Smem<R, T>::kCoefWords;
  const int state_words = Smem<R, T>::kStateWords;
  const int front = coef_words + 2 * T * p.rec_words;
  uint32_t* rawbuf = smem + coef_words;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + ((max(front, state_words) + 3) & ~3));
  __shared__ int s_abort;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned raw_bytes = (unsigned)(T * p.rec_words * 4);
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  __syncthreads();
  // per raw buffer: bulk copies issued and waited for (identical in every thread)
  unsigned issued[2] = {0u, 0u}, waited[2] = {0u, 0u};

  for (unsigned long long item = blockIdx.x; item < p.total_items; item += gridDim.x) {
    int b = 0;
    while (b + 1 < p.nblocks && p.blocks[b + 1].item_begin <= item) b++;
    const BlockDesc& bd = p.blocks[b];
    const unsigned long long local = item - bd.item_begin;
    const uint32_t o = odd_bits(bd.g_base) | (uint32_t)(local & ((1ull << bd.no_free) - 1));
    const uint32_t chunk = (uint32_t)(local >> bd.no_free);
    const int nroles = (int)bd.nroles;
    const uint32_t ehigh = even_bits(bd.g_base) | (chunk << nroles);

    uint32_t tmax[P], m1[P], ts[P];
#pragma unroll
    for (int v = 0; v < P; v++) tmax[v] = m1[v] = ts[v] = 0u;

    if (tid == 0) bulk_load(rawbuf, p.rec, raw_bytes, &bars[0]);
    issued[0]++;
    if (p.ntiles > 1) {
      if (tid == 0) bulk_load(rawbuf + T * p.rec_words, p.rec + (size_t)T * p.rec_words, raw_bytes, &bars[1]);
      issued[1]++;
    }

    for (int t = 0; t < p.ntiles; t++) {
      const int buf = t & 1;
      uint32_t* cbuf = coefbuf + buf * T * kCStride;
      // ---- producer: one thread per conformation of the tile
      if (tid < T) {
        if (!mbar_wait(&bars[buf], waited[buf] & 1u)) {
          atomicOr(p.err, kErrTimeout);
          s_abort = 1;
        } else {
          const uint32_t* r = rawbuf + buf * T * p.rec_words + tid * p.rec_words;
          uint32_t* c = cbuf + tid * kCStride;
          const int s = t * T + tid;
          if (s < p.S_dir) {
            uint32_t a[NROLE];
#pragma unroll
            for (int k = 0; k < NROLE; k++) a[k] = k < nroles ? 2u * coef(r[k], o) : 0u;
            uint32_t extra = 0;
            for (int k = nroles; k < p.NE; k++)
              if ((ehigh >> k) & 1u) extra += coef(r[k], o);
            const uint32_t base = 2u * (odd_part(r, p.NE, o) + extra + 1u);
            const uint32_t split_hi = a[0] << 16;
            // lane table: base + subset sums of the 5 lane coefficients, packed
            uint32_t lt[32];
            lt[0] = base;
#pragma unroll
            for (int l = 1; l < 32; l++) {
              const int hb = 31 - __clz(l);
              lt[l] = lt[l ^ (1 << hb)] + a[R + hb];
            }
#pragma unroll
            for (int l = 0; l < 32; l += 4)
              *reinterpret_cast<uint4*>(c + l) = make_uint4(lt[l] * 0x10001u + split_hi, lt[l + 1] * 0x10001u + split_hi,
                                                            lt[l + 2] * 0x10001u + split_hi, lt[l + 3] * 0x10001u + split_hi);
            uint32_t wt[8];
            wt[0] = 0;
#pragma unroll
            for (int w = 1; w < 8; w++) {
              const int hb = 31 - __clz(w);
              wt[w] = wt[w ^ (1 << hb)] + a[R + kLaneRoles + hb];
            }
            *reinterpret_cast<uint4*>(c + 32) = make_uint4(wt[0] * 0x10001u, wt[1] * 0x10001u, wt[2] * 0x10001u, wt[3] * 0x10001u);
            *reinterpret_cast<uint4*>(c + 36) = make_uint4(wt[4] * 0x10001u, wt[5] * 0x10001u, wt[6] * 0x10001u, wt[7] * 0x10001u);
            uint32_t tp[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int j = 0; j < R - 1; j++) tp[j] = a[1 + j] * 0x10001u;
            *reinterpret_cast<uint4*>(c + 40) = make_uint4(tp[0], tp[1], tp[2], tp[3]);
            *reinterpret_cast<uint4*>(c + 44) = make_uint4(tp[4], tp[5], tp[6], tp[7]);
          } else {
            // padding conformation: every score 0, below every real (biased) score
#pragma unroll
            for (int k = 0; k < 48; k += 4) *reinterpret_cast<uint4*>(c + k) = make_uint4(0, 0, 0, 0);
          }
        }
      }
      waited[buf]++;
      __syncthreads();
      if (s_abort) break;
      // raw[buf] has been read by every producer: prefetch tile t + 2 into it
      if (t + 2 < p.ntiles) {
        if (tid == 0)
          bulk_load(rawbuf + buf * T * p.rec_words, p.rec + (size_t)(t + 2) * T * p.rec_words, raw_bytes, &bars[buf]);
        issued[buf]++;
      }

      // ---- consumer: every thread, every conformation of the tile
#pragma unroll 2
      for (int s = 0; s < T; s++) {
        const uint32_t* cs = cbuf + s * kCStride;
        const uint32_t b0 = cs[lane] + cs[32 + warp];
        uint32_t tpv[8];
        {
          const uint4 q0 = *reinterpret_cast<const uint4*>(cs + 40);
          tpv[0] = q0.x; tpv[1] = q0.y; tpv[2] = q0.z; tpv[3] = q0.w;
          if (R - 1 > 4) {
            const uint4 q1 = *reinterpret_cast<const uint4*>(cs + 44);
            tpv[4] = q1.x; tpv[5] = q1.y; tpv[6] = q1.z; tpv[7] = q1.w;
          }
        }
        uint32_t x[P];
        x[0] = b0;
#pragma unroll
        for (int v = 1; v < P; v++) {
          const int hb = 31 - __clz(v);
          x[v] = x[v ^ (1 << hb)] + tpv[hb];
        }
#pragma unroll
        for (int v = 0; v < P; v++) tmax[v] = vmax2(tmax[v], x[v]);
      }
      // ---- tile merge: best (doubled) with tie bit, and first tile reaching it
      const uint32_t tpk = (uint32_t)t * 0x10001u;
#pragma unroll
      for (int v = 0; v < P; v++) {
        const uint32_t mb = m1[v] & 0xFFFEFFFEu;
        const uint32_t gt = __vcmpgtu2(tmax[v], m1[v]);
        const uint32_t eq = __vcmpeq2(tmax[v], mb);
        m1[v] = (gt & tmax[v]) | (~gt & (m1[v] | (eq & 0x00010001u)));
        ts[v] = (gt & tpk) | (~gt & ts[v]);
        tmax[v] = 0u;
      }
    }
    if (s_abort) break;
    __syncthreads();  // every warp is done with the coefficient buffers

    // ---- epilogue: park the state in shared memory, resolve candidates per warp
    uint32_t* st_best = smem;                 // [P][kThreads]
    uint32_t* st_tile = smem + P * kThreads;  // [P][kThreads]
#pragma unroll
    for (int v = 0; v < P; v++) {
      st_best[v * kThreads + tid] = m1[v];
      st_tile[v * kThreads + tid] = ts[v];
    }
    const bool want_aux = p.aux != nullptr;
    const uint32_t role_hi = ((uint32_t)lane << R) | ((uint32_t)warp << (R + kLaneRoles));
    const uint32_t role_mask = (1u << nroles) - 1u;
    for (int v = 0; v < P; v++) {
      const uint32_t mine_best = st_best[v * kThreads + tid];
      const uint32_t mine_tile = st_tile[v * kThreads + tid];
      int ph[2] = {-1, -1}, ax[2] = {-1, -1};
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const uint32_t field = (mine_best >> (16 * h)) & 0xFFFFu;
        const uint32_t rw = (uint32_t)h | ((uint32_t)v << 1) | role_hi;
        const bool valid = nroles >= NROLE || (rw >> nroles) == 0u;
        const bool cand = valid && field > 1u && (want_aux || !(field & 1u));
        uint32_t mask = __ballot_sync(0xFFFFFFFFu, cand);
        while (mask) {
          const int src = __ffs(mask) - 1;
          mask &= mask - 1;
          const uint32_t sfield = __shfl_sync(0xFFFFFFFFu, field, src);
          const int tile = (int)((__shfl_sync(0xFFFFFFFFu, mine_tile, src) >> (16 * h)) & 0xFFFFu);
          const uint32_t rws = (uint32_t)h | ((uint32_t)v << 1) | ((uint32_t)src << R) | ((uint32_t)warp << (R + kLaneRoles));
          const uint32_t eall = (rws & role_mask) | ehigh;
          const uint32_t want = sfield & 0xFFFEu;
          int count = 0, first = -1;
          for (int i = 0; i < T; i += 32) {
            const int s = tile * T + i + lane;
            bool match = false;
            if (s < p.S_dir) {
              const uint32_t* r = p.rec + (size_t)s * p.rec_words;
              uint32_t x = odd_part(r, p.NE, o);
              for (uint32_t e = eall; e; e &= e - 1) x += coef(r[__ffs(e) - 1], o);
              match = 2u * (x + 1u) == want;
            }
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, match);
            if (first < 0 && bal) first = tile * T + i + __ffs(bal) - 1;
            count += __popc(bal);
          }
          if (lane == src) {
            ax[h] = first >= 0 ? p.conf_class[first] : -1;
            ph[h] = (!(sfield & 1u) && count == 1) ? ax[h] : -1;
          }
        }
      }
      // write the two sequences of this packed register (ids differ in bit 0)
      const uint32_t rw0 = ((uint32_t)v << 1) | role_hi;
      const bool valid0 = nroles >= NROLE || (rw0 >> nroles) == 0u;
      const bool valid1 = nroles >= NROLE || ((rw0 | 1u) >> nroles) == 0u;
      if (valid0) {
        const uint32_t e0 = (rw0 & role_mask) | ehigh;
        const unsigned long long g0 = interleave(e0, o);
        const unsigned long long idx = bd.out_off + (g0 - bd.g_base);
        const bool pair_ok = valid1 && ((reinterpret_cast<uintptr_t>(p.phen + idx) & 7u) == 0u) &&
                             (!want_aux || (reinterpret_cast<uintptr_t>(p.aux + idx) & 7u) == 0u);
        if (pair_ok) {
          *reinterpret_cast<int2*>(p.phen + idx) = make_int2(ph[0], ph[1]);
          if (want_aux) *reinterpret_cast<int2*>(p.aux + idx) = make_int2(ax[0], ax[1]);
        } else {
          p.phen[idx] = ph[0];
          if (want_aux) p.aux[idx] = ax[0];
          if (valid1) {
            p.phen[idx + 1] = ph[1];
            if (want_aux) p.aux[idx + 1] = ax[1];
          }
        }
      }
    }
    __syncthreads();  // state area is reused as coefficient buffers by the next item
  }
  // after an abort, wait (bounded) for bulk copies still in flight before exiting
  if (tid == 0) {
    for (int k = 0; k < 2; k++)
      while (waited[k] < issued[k]) {
        if (!mbar_wait(&bars[k], waited[k] & 1u)) break;
        waited[k]++;
      }
  }
}

template <int R, int T>
size_t smem_bytes(int rec_words) {
  const size_t front = (size_t)Smem<R, T>::kCoefWords + 2ull * T * rec_words;
  const size_t words = std::max(front, (size_t)Smem<R, T>::kStateWords);
  return (((words + 3) & ~(size_t)3) * 4) + 2 * sizeof(uint64_t);
}

template <int R, int T>
int launch(const Params& prm, cudaStream_t stream) {
  const size_t smem = smem_bytes<R, T>(prm.rec_words);
  auto kern = phenotype_kernel<R, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return hp::cuda_fail(e, "cudaFuncSetAttribute(phenotype_kernel)");
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (e != cudaSuccess) return hp::cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (per_sm < 1) return hp::fail(HP_EUNSUPPORTED, "phenotype kernel does not fit on this GPU");
  unsigned long long grid = (unsigned long long)sms * per_sm;
  if (grid > prm.total_items) grid = prm.total_items;
  kern<<<(unsigned)grid, kThreads, smem, stream>>>(prm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return hp::cuda_fail(e, "phenotype_kernel launch");
  return HP_OK;
}

}  // namespace

namespace hp {

// Split [begin, begin + count) into aligned power-of-two blocks and fill the
// launch descriptors for a kernel with R register bits.
int plan_blocks(const hp_structs* s, unsigned long long begin, unsigned long long count, int R, Params& prm) {
  const int nrole_max = R + kLaneRoles + kWarpRoles;
  unsigned long long pos = begin, end = begin + count, items = 0;
  int nb = 0;
  while (pos < end) {
    int m = 0;
    while (m < 63) {
      const unsigned long long size = 1ull << (m + 1);
      if ((pos & (size - 1)) != 0 || pos + size > end) break;
      m++;
    }
    if (nb >= kMaxBlocks) return fail(HP_EUNSUPPORTED, "sequence range splits into too many aligned blocks");
    BlockDesc& d = prm.blocks[nb++];
    d.g_base = pos;
    d.out_off = pos - begin;
    d.item_begin = items;
    d.ne_free = (unsigned)std::min((m + 1) / 2, s->NE);
    d.no_free = (unsigned)std::min(m / 2, s->NO);
    d.nroles = (unsigned)std::min((int)d.ne_free, nrole_max);
    d.pad = 0;
    const unsigned chunk_bits = d.ne_free - d.nroles;
    items += (1ull << d.no_free) << chunk_bits;
    pos += 1ull << m;
  }
  prm.nblocks = nb;
  prm.total_items = items;
  return HP_OK;
}

}  // namespace hp

extern "C" int hp_phenotype_map(const hp_structs* s, uint64_t seq_begin, uint64_t seq_count, int32_t gap_threshold,
                                int32_t* d_phen, int32_t* d_argmin_aux, void* stream) {
  if (!s) return hp::fail(HP_EINVAL, "hp_phenotype_map: library is NULL");
  if (!d_phen) return hp::fail(HP_EINVAL, "hp_phenotype_map: d_phen is NULL");
  if (gap_threshold != 1) return hp::fail(HP_EUNSUPPORTED, "hp_phenotype_map: only gap_threshold 1 is implemented");
  if (s->N > 2 * hp::kMaxHalf) return hp::fail(HP_EUNSUPPORTED, "hp_phenotype_map: N > 40");
  const unsigned long long space = s->N >= 64 ? ~0ull : (1ull << s->N);
  if (seq_count == 0) return HP_OK;
  if (seq_begin >= space || seq_count > space - seq_begin)
    return hp::fail(HP_EINVAL, "hp_phenotype_map: sequence range exceeds 2^N");
  hp::DevTables* dt = nullptr;
  int rc = hp::device_tables(s, &dt);
  if (rc != HP_OK) return rc;
  constexpr int R = 6, T = 256;
  static_assert(T % 4 == 0 && hp::kRecPad % T == 0, "tiles must tile the padded record table");
  Params* prm = new (std::nothrow) Params();
  if (!prm) return hp::fail(HP_ENOMEM, "hp_phenotype_map: out of host memory");
  prm->rec = dt->rec;
  prm->conf_class = dt->conf_class;
  prm->phen = d_phen;
  prm->aux = d_argmin_aux;
  prm->S_dir = s->S_dir;
  prm->ntiles = (s->S_dir + T - 1) / T;
  prm->rec_words = s->rec_words;
  prm->NE = s->NE;
  prm->NO = s->NO;
  rc = hp::plan_blocks(s, seq_begin, seq_count, R, *prm);
  if (rc != HP_OK) {
    delete prm;
    return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned int* err = nullptr;
  cudaError_t e = cudaMallocAsync(&err, sizeof(unsigned int), st);
  if (e != cudaSuccess) {
    delete prm;
    return hp::cuda_fail(e, "cudaMallocAsync(error word)");
  }
  cudaMemsetAsync(err, 0, sizeof(unsigned int), st);
  prm->err = err;
  rc = launch<R, T>(*prm, st);
  delete prm;
  unsigned int herr = 0;
  if (rc == HP_OK) {
    e = cudaMemcpyAsync(&herr, err, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_phenotype_map: kernel execution");
  }
  cudaFreeAsync(err, st);
  if (rc == HP_OK && (herr & kErrTimeout)) rc = hp::fail(HP_ETIMEOUT, "hp_phenotype_map: a bulk-copy wait timed out");
  return rc;
}
