// Per-sequence ground-state scan for arbitrary sequence ids, with optional
// exact bound pruning seeded by candidate conformations (the learned proposal).
//
// One warp scans one sequence against every conformation.  The score of a
// sequence h on conformation s is x = 10 A + 3 B (the negated Eq. 1 energy,
// Table 1 x 10), with A = sum_i h_i c_i(s) (contacts touching an H) and
// B = #HH contacts.  Because B <= C and 2B <= A,
//     x <= U(A) = 10 A + 3 min(C, floor(A / 2)),
// so with a candidate score x_cand (the best exact score among the candidate
// conformations, a lower bound on the true best) every conformation with
// U(A_s(h)) < x_cand can neither be the minimum nor tie it and is skipped.
// The same test on per-tile maxima of the contact counts (conformations sorted
// by their contact-count vectors, so tiles are homogeneous) skips whole tiles:
// the lanes test 32 tiles at once and the warp visits the survivors.  Skips are
// strict, so the phenotype, the tie status and the lowest-index minimiser are
// exactly those of the full scan.
//
// Tables are word-major inside each 128-conformation tile (the six count
// bit-planes, then the NE contact masks, each as 128 consecutive words), so
// the lanes' loads for their four conformations of a tile are coalesced.
//
// Reductions use warp primitives: running best / count / first index per lane,
// then __reduce_max_sync, __reduce_add_sync and __reduce_min_sync.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "hp_internal.h"

namespace {

constexpr int kScanTile = 128;   // conformations per bound tile
constexpr int kScanWarps = 8;    // warps (sequences in flight) per CTA

struct ScanParams {
  const uint32_t* soa;       // scan-order tables, (6 + NE) x 128 words per tile
  const int32_t* idx;        // original index of each scan-order record (-1 padding)
  const uint32_t* tb;        // per tile: [0..2] even-residue max-count masks, [3..5] odd-residue ones
  const uint32_t* orig_rec;  // original-order records (candidates)
  const int32_t* conf_class;
  const unsigned long long* ids;
  const int32_t* cand;       // n x k original conformation indices (-1: none) or NULL
  int32_t* phen;
  int32_t* aux;
  unsigned long long* counters;  // [0] conformations evaluated exactly, [1] bounds evaluated
  long long n;
  int k, rec_words, NE, C, S_dir, ntiles, prune;
};

__device__ __forceinline__ uint32_t even_of(unsigned long long g) {
  uint32_t r = 0;
#pragma unroll
  for (int k = 0; k < hp::kMaxHalf; k++) r |= (uint32_t)((g >> (2 * k)) & 1ull) << k;
  return r;
}
__device__ __forceinline__ uint32_t odd_of(unsigned long long g) {
  uint32_t r = 0;
#pragma unroll
  for (int k = 0; k < hp::kMaxHalf; k++) r |= (uint32_t)((g >> (2 * k + 1)) & 1ull) << k;
  return r;
}

// A = sum_i h_i c_i from bit-planes of the even (we) and odd (wo) contact counts
__device__ __forceinline__ int weight_sum(uint32_t e, uint32_t o, const uint32_t* we, const uint32_t* wo) {
  return (__popc(e & __ldg(we)) + __popc(o & __ldg(wo))) + 2 * (__popc(e & __ldg(we + 1)) + __popc(o & __ldg(wo + 1))) +
         4 * (__popc(e & __ldg(we + 2)) + __popc(o & __ldg(wo + 2)));
}
__device__ __forceinline__ int upper(int A, int C) { return 10 * A + 3 * min(C, A >> 1); }

// A of one conformation from its six word-major count planes (c points at its tile slot)
__device__ __forceinline__ int count_sum(uint32_t e, uint32_t o, const uint32_t* c) {
  constexpr int T = kScanTile;
  return (__popc(e & __ldg(c)) + __popc(o & __ldg(c + 3 * T))) + 2 * (__popc(e & __ldg(c + T)) + __popc(o & __ldg(c + 4 * T))) +
         4 * (__popc(e & __ldg(c + 2 * T)) + __popc(o & __ldg(c + 5 * T)));
}

// exact score of (e, o) on one record
__device__ __forceinline__ int score_of(const uint32_t* r, int NE, uint32_t e, uint32_t o, int A) {
  int B = 0;
  for (uint32_t m = e; m; m &= m - 1) B += __popc(o & __ldg(r + (__ffs(m) - 1)));
  return 10 * A + 3 * B;
}

__global__ void __launch_bounds__(32 * kScanWarps, 4) seq_scan_kernel(const ScanParams p) {
  const int lane = threadIdx.x & 31;
  const long long warps_total = (long long)gridDim.x * kScanWarps;
  const size_t tile_words = (size_t)(6 + p.NE) * kScanTile;
  unsigned long long n_exact = 0, n_bound = 0;
  for (long long q = (long long)blockIdx.x * kScanWarps + (threadIdx.x >> 5); q < p.n; q += warps_total) {
    const unsigned long long g = p.ids[q];
    const uint32_t e = even_of(g), o = odd_of(g);
    // candidate score: best exact score over the candidate conformations
    int cand = -1;
    if (p.prune && p.cand) {
      int best = -1;
      for (int j = lane; j < p.k; j += 32) {
        const int s = p.cand[q * p.k + j];
        if (s >= 0 && s < p.S_dir) {
          const uint32_t* r = p.orig_rec + (size_t)s * p.rec_words;
          const int A = weight_sum(e, o, r + p.NE + 3, r + p.NE);
          best = max(best, score_of(r, p.NE, e, o, A));
        }
      }
      cand = __reduce_max_sync(0xFFFFFFFFu, best);
    }
    int best = -1, cnt = 0, first = INT_MAX;
    for (int t0 = 0; t0 < p.ntiles; t0 += 32) {
      // lane l tests tile t0 + l
      const int tl = t0 + lane;
      bool keep = tl < p.ntiles;
      if (keep && cand >= 0) {
        const uint32_t* tb = p.tb + (size_t)tl * 8;
        keep = upper(weight_sum(e, o, tb, tb + 3), p.C) >= cand;
      }
      for (uint32_t kept = __ballot_sync(0xFFFFFFFFu, keep); kept; kept &= kept - 1) {
        const int t = t0 + __ffs(kept) - 1;
        const uint32_t* base = p.soa + (size_t)t * tile_words;
        // two conformations per lane at a time; every load of a pair is independent of the
        // others, so they are all in flight together
#pragma unroll
        for (int r = 0; r < kScanTile / 32; r += 2) {
          const int i0 = lane + 32 * r, i1 = i0 + 32;
          const int orig0 = __ldg(p.idx + t * kScanTile + i0), orig1 = __ldg(p.idx + t * kScanTile + i1);
          const uint32_t* c0 = base + i0;
          const uint32_t* c1 = base + i1;
          const int A0 = count_sum(e, o, c0), A1 = count_sum(e, o, c1);
          const bool need0 = orig0 >= 0 && (cand < 0 || upper(A0, p.C) >= cand);
          const bool need1 = orig1 >= 0 && (cand < 0 || upper(A1, p.C) >= cand);
          n_bound += (orig0 >= 0) + (orig1 >= 0);
          if (!__any_sync(0xFFFFFFFFu, need0 || need1)) continue;
          // B = sum over the H even residues k of #H odd neighbours (mask word 6 + k); e is the
          // same for the whole warp, so the bit tests are uniform
          int B0 = 0, B1 = 0;
#pragma unroll
          for (int k = 0; k < hp::kMaxHalf; k++) {
            if ((e >> k) & 1u) {
              const uint32_t w0 = need0 ? __ldg(c0 + (6 + k) * kScanTile) : 0u;
              const uint32_t w1 = need1 ? __ldg(c1 + (6 + k) * kScanTile) : 0u;
              B0 += __popc(o & w0);
              B1 += __popc(o & w1);
            }
          }
          if (need0) {
            const int x = 10 * A0 + 3 * B0;
            n_exact++;
            if (x > best) {
              best = x;
              cnt = 1;
              first = orig0;
            } else if (x == best) {
              cnt++;
              first = min(first, orig0);
            }
          }
          if (need1) {
            const int x = 10 * A1 + 3 * B1;
            n_exact++;
            if (x > best) {
              best = x;
              cnt = 1;
              first = orig1;
            } else if (x == best) {
              cnt++;
              first = min(first, orig1);
            }
          }
        }
      }
    }
    const int M = __reduce_max_sync(0xFFFFFFFFu, best);
    const int total = __reduce_add_sync(0xFFFFFFFFu, best == M ? cnt : 0);
    const int f = __reduce_min_sync(0xFFFFFFFFu, best == M ? first : INT_MAX);
    if (lane == 0) {
      const int cls = (f >= 0 && f < p.S_dir) ? __ldg(p.conf_class + f) : -1;
      p.phen[q] = (total == 1 || p.S_dir == 1) ? cls : -1;
      if (p.aux) p.aux[q] = cls;
    }
  }
  if (p.counters) {
    for (int off = 16; off; off >>= 1) {
      n_exact += __shfl_xor_sync(0xFFFFFFFFu, n_exact, off);
      n_bound += __shfl_xor_sync(0xFFFFFFFFu, n_bound, off);
    }
    if (lane == 0) {
      atomicAdd(p.counters, n_exact);
      atomicAdd(p.counters + 1, n_bound);
    }
  }
}

}  // namespace

namespace hp {

// Scan order: conformations sorted by their vector of per-residue contact
// counts (lexicographic), so consecutive ones expose similar residues and the
// per-tile maxima of the counts stay close to each member's counts.
int scan_tables(const hp_structs* cs, DevTables** out) {
  DevTables* dt = nullptr;
  int rc = device_tables(cs, &dt);
  if (rc != HP_OK) return rc;
  hp_structs* s = const_cast<hp_structs*>(cs);
  std::lock_guard<std::mutex> lock(s->mu);
  if (dt->scan_soa) {
    *out = dt;
    return HP_OK;
  }
  const int N = s->N, NE = s->NE, W = s->rec_words;
  const size_t spad = ((size_t)s->S_dir + kRecPad - 1) / kRecPad * kRecPad;
  std::vector<std::vector<uint8_t>> cvec((size_t)s->S_dir, std::vector<uint8_t>(N, 0));
  for (int32_t c = 0; c < s->S_dir; c++)
    for (int k = 0; k < s->C; k++) {
      cvec[c][s->contacts[((size_t)c * s->C + k) * 2]]++;
      cvec[c][s->contacts[((size_t)c * s->C + k) * 2 + 1]]++;
    }
  std::vector<int32_t> order((size_t)s->S_dir);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cvec[a] < cvec[b]; });
  // word-major tiles: count planes (even residues bits 0..2 = record words NE+3..NE+5, odd
  // residues = NE..NE+2), then the NE contact masks (record words 0..NE-1)
  const int TW = 6 + NE;
  const int ntiles = (int)(spad / kScanTile);
  std::vector<uint32_t> soa((size_t)ntiles * TW * kScanTile, 0u);
  std::vector<int32_t> idx(spad, -1);
  for (size_t j = 0; j < order.size(); j++) {
    const uint32_t* r = s->rec.data() + (size_t)order[j] * W;
    uint32_t* t = soa.data() + (j / kScanTile) * TW * kScanTile + (j % kScanTile);
    for (int b = 0; b < 3; b++) {
      t[(size_t)b * kScanTile] = r[NE + 3 + b];
      t[(size_t)(3 + b) * kScanTile] = r[NE + b];
    }
    for (int k = 0; k < NE; k++) t[(size_t)(6 + k) * kScanTile] = r[k];
    idx[j] = order[j];
  }
  std::vector<uint32_t> tb((size_t)ntiles * 8, 0u);
  for (int t = 0; t < ntiles; t++) {
    uint8_t cmax[kMaxN] = {0};
    for (int j = t * kScanTile; j < (t + 1) * kScanTile && j < s->S_dir; j++)
      for (int i = 0; i < N; i++) cmax[i] = std::max(cmax[i], cvec[order[j]][i]);
    for (int i = 0; i < N; i++)
      for (int b = 0; b < 3; b++)
        if ((cmax[i] >> b) & 1) tb[(size_t)t * 8 + ((i & 1) ? 3 : 0) + b] |= 1u << (i / 2);
  }
  cudaError_t e = cudaMalloc(&dt->scan_soa, soa.size() * 4);
  if (e == cudaSuccess) e = cudaMalloc(&dt->scan_idx, idx.size() * 4);
  if (e == cudaSuccess) e = cudaMalloc(&dt->scan_tb, tb.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(dt->scan_soa, soa.data(), soa.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dt->scan_idx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dt->scan_tb, tb.data(), tb.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dt->scan_soa);
    cudaFree(dt->scan_idx);
    cudaFree(dt->scan_tb);
    dt->scan_soa = nullptr;
    dt->scan_idx = nullptr;
    dt->scan_tb = nullptr;
    return cuda_fail(e, "per-sequence scan tables");
  }
  dt->scan_tile = kScanTile;
  *out = dt;
  return HP_OK;
}

}  // namespace hp

extern "C" int hp_sequence_scan(const hp_structs* s, const uint64_t* d_ids, int64_t n, const int32_t* d_cand,
                                int32_t k, int32_t* d_phen, int32_t* d_aux, uint64_t* d_counters, void* stream) {
  if (!s || !d_ids || !d_phen) return hp::fail(HP_EINVAL, "hp_sequence_scan: NULL argument");
  if (n < 0 || k < 0 || (d_cand && k == 0)) return hp::fail(HP_EINVAL, "hp_sequence_scan: bad sizes");
  if (s->N > 2 * hp::kMaxHalf) return hp::fail(HP_EUNSUPPORTED, "hp_sequence_scan: N > 40");
  if (n == 0) return HP_OK;
  hp::DevTables* dt = nullptr;
  int rc = hp::scan_tables(s, &dt);
  if (rc != HP_OK) return rc;
  ScanParams p;
  p.soa = dt->scan_soa;
  p.idx = dt->scan_idx;
  p.tb = dt->scan_tb;
  p.orig_rec = dt->rec;
  p.conf_class = dt->conf_class;
  p.ids = reinterpret_cast<const unsigned long long*>(d_ids);
  p.cand = d_cand;
  p.phen = d_phen;
  p.aux = d_aux;
  p.counters = reinterpret_cast<unsigned long long*>(d_counters);
  p.n = n;
  p.k = k;
  p.rec_words = s->rec_words;
  p.NE = s->NE;
  p.C = s->C;
  p.S_dir = s->S_dir;
  p.ntiles = (int)((((size_t)s->S_dir + hp::kRecPad - 1) / hp::kRecPad * hp::kRecPad) / kScanTile);
  p.prune = d_cand != nullptr;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (n + kScanWarps - 1) / kScanWarps;
  blocks = std::min<long long>(blocks, (long long)sms * 8);
  seq_scan_kernel<<<(unsigned)blocks, 32 * kScanWarps, 0, (cudaStream_t)stream>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_sequence_scan: launch");
  return HP_OK;
}
