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
// Skips are strict, so the phenotype, the tie status and the lowest-index
// minimiser are exactly those of the full scan.
//
// A depends on a conformation only through its contact-count vector c(s), and
// many conformations share one (3x3x3: 103,346 conformations, 6,291 vectors).
// Conformations are therefore sorted by c(s) and scanned group by group (a
// group = a run of equal vectors): the lanes compute A and the bound for 32
// groups at once, a warp prefix sum lays the members of the groups that
// survive end to end, and each lane takes one member per round, finds its
// group by a shuffle binary search and adds only B (its contact masks of the H
// even residues).  Without a candidate score there is nothing to prune and
// the members are scanned directly, two per lane at a time with A from their
// own count planes.  Tables are word-major (count planes by group and by
// member, masks by member), so the lanes' loads are coalesced.
//
// Reductions use warp primitives: running best / count / first index per lane,
// then __reduce_max_sync, __reduce_add_sync and __reduce_min_sync.
//
// Energy-gap threshold T >= 1 (Section 2.1; the Appendix C kernel keeps the
// lowest and second-lowest energy): a sequence folds iff E2 - E1 >= T, E2 the
// second-lowest energy counted with multiplicity.  The kernel variant with
// GAP set also keeps each lane's second-best score; pruning then skips only
// groups with U(A) <= x_cand - T, whose every conformation lies at least T
// below the best score, so the phenotype stays exact and the gap is exact
// below T (it is reported clipped at T when pruning).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "hp_internal.h"

namespace {

constexpr int kScanWarps = 8;      // warps (sequences in flight) per CTA
constexpr int kClusterGroups = 8;  // groups per cluster (four clusters per warp step)

struct ScanParams {
  const uint32_t* gcnt;      // 6 x gpad count planes per group (even bits 0..2, odd bits 0..2)
  const uint32_t* ccnt;      // 12 x cpad planes per cluster of kClusterGroups groups: the componentwise
                             // minimum of its count vectors (6), the maximum excess over it (6)
  const int32_t* cl1;        // cpad: per cluster the largest L1 excess of a member group over the minimum
  const int32_t* gbeg;       // ngroups + 1 member ranges
  const uint32_t* mcnt;      // 6 x spad count planes per member (the unpruned scan)
  const uint32_t* mmask;     // NE x spad contact masks per member
  const int32_t* midx;       // original index per member
  const uint32_t* orig_rec;  // original-order records (candidates)
  const int32_t* conf_class;
  const unsigned long long* ids;  // n sequence ids
  const int32_t* cand;       // n x k original conformation indices (-1: none) or NULL
  int32_t* phen;
  int32_t* aux;
  int32_t* gap;              // n energy gaps E2 - E1 or NULL (GAP variant)
  unsigned long long* counters;  // [0] conformations evaluated exactly, [1] group bounds evaluated
  long long n;
  int k, rec_words, NE, C, S_dir, ngroups, gpad, spad, prune, nclusters, cpad;
  int T;                     // energy-gap threshold (1 unless GAP)
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

// exact score of (e, o) on one record
__device__ __forceinline__ int score_of(const uint32_t* r, int NE, uint32_t e, uint32_t o, int A) {
  int B = 0;
  for (uint32_t m = e; m; m &= m - 1) B += __popc(o & __ldg(r + (__ffs(m) - 1)));
  return 10 * A + 3 * B;
}

template <bool GAP>
__global__ void __launch_bounds__(32 * kScanWarps, 4) seq_scan_kernel(const ScanParams p) {
  const int lane = threadIdx.x & 31;
  const long long warps_total = (long long)gridDim.x * kScanWarps;
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
    // a group survives when its bound reaches cut (T = 1: the candidate score itself)
    const int cut = GAP ? cand - p.T + 1 : cand;
    int best = -1, cnt = 0, first = INT_MAX;
    int sec = -1;  // GAP: best score of this lane's conformations other than one at `best`
    auto take = [&](int x, int orig) {
      n_exact++;
      if (x > best) {
        if (GAP) sec = best;
        best = x;
        cnt = 1;
        first = orig;
      } else if (x == best) {
        cnt++;
        first = min(first, orig);
        if (GAP) sec = best;
      } else if (GAP) {
        sec = max(sec, x);
      }
    };
    if (cand < 0) {
      // nothing to prune with: every member, two per lane at a time, A from its own count planes
      for (int m0 = 0; m0 < p.S_dir; m0 += 64) {
        const int m[2] = {m0 + lane, m0 + 32 + lane};
        int A[2], B[2] = {0, 0}, orig[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
          const int mm = min(m[u], p.spad - 1);
          const uint32_t* c = p.mcnt + mm;
          const size_t w = (size_t)p.spad;
          A[u] = (__popc(e & __ldg(c)) + __popc(o & __ldg(c + 3 * w))) +
                 2 * (__popc(e & __ldg(c + w)) + __popc(o & __ldg(c + 4 * w))) +
                 4 * (__popc(e & __ldg(c + 2 * w)) + __popc(o & __ldg(c + 5 * w)));
          orig[u] = m[u] < p.S_dir ? __ldg(p.midx + mm) : -1;
        }
#pragma unroll
        for (int k = 0; k < hp::kMaxHalf; k++)
          if ((e >> k) & 1u) {
#pragma unroll
            for (int u = 0; u < 2; u++) B[u] += __popc(o & __ldg(p.mmask + (size_t)k * p.spad + min(m[u], p.spad - 1)));
          }
#pragma unroll
        for (int u = 0; u < 2; u++)
          if (orig[u] >= 0) take(10 * A[u] + 3 * B[u], orig[u]);
      }
    }
    // the next surviving cluster's count planes and member ranges are loaded while the current
    // ones are tested (the step is short and latency-bound otherwise)
    uint32_t cw[6] = {0, 0, 0, 0, 0, 0};
    int cb0 = 0, cb1 = 0;
    auto fetch = [&](int gi, uint32_t (&c)[6], int& b0, int& b1) {
      if (gi >= 0 && gi < p.ngroups) {
#pragma unroll
        for (int k = 0; k < 6; k++) c[k] = __ldg(p.gcnt + (size_t)k * p.gpad + gi);
        b0 = __ldg(p.gbeg + gi);
        b1 = __ldg(p.gbeg + gi + 1);
      }
    };
    // Groups come in clusters of kClusterGroups.  With m the componentwise minimum of a
    // cluster's count vectors, d its largest excess over m and L its largest L1 excess, every
    // group's A = h.m + h.(c - m) <= h.m + min(h.d, L) (h in {0,1}^N), so when the bound of that
    // value falls below cut the whole cluster is skipped.  The lanes test 32 clusters at once;
    // pop_cluster walks the survivors and a warp step takes four of them (lane l: cluster l / 8,
    // group l % 8).
    int k0 = -32;
    uint32_t sv = 0;
    auto pop_cluster = [&]() -> int {
      while (sv == 0) {
        k0 += 32;
        if (k0 >= p.nclusters) return -1;
        const int ki = k0 + lane;
        bool keep = false;
        if (ki < p.nclusters) {
          uint32_t c[12];
#pragma unroll
          for (int k = 0; k < 12; k++) c[k] = __ldg(p.ccnt + (size_t)k * p.cpad + ki);
          const int Am = (__popc(e & c[0]) + __popc(o & c[3])) + 2 * (__popc(e & c[1]) + __popc(o & c[4])) +
                         4 * (__popc(e & c[2]) + __popc(o & c[5]));
          const int Ad = (__popc(e & c[6]) + __popc(o & c[9])) + 2 * (__popc(e & c[7]) + __popc(o & c[10])) +
                         4 * (__popc(e & c[8]) + __popc(o & c[11]));
          n_bound++;
          keep = upper(Am + min(Ad, __ldg(p.cl1 + ki)), p.C) >= cut;
        }
        sv = __ballot_sync(0xFFFFFFFFu, keep);
      }
      const int cl = k0 + __ffs(sv) - 1;
      sv &= sv - 1;
      return cl;
    };
    // this lane's group of the next step (-1: none); false when no cluster is left
    auto next_step = [&](int& gi) -> bool {
      const int c0 = pop_cluster(), c1 = c0 >= 0 ? pop_cluster() : -1, c2 = c1 >= 0 ? pop_cluster() : -1,
                c3 = c2 >= 0 ? pop_cluster() : -1;
      const int q = lane / kClusterGroups, mine = q == 0 ? c0 : q == 1 ? c1 : q == 2 ? c2 : c3;
      gi = mine >= 0 ? mine * kClusterGroups + lane % kClusterGroups : -1;
      return c0 >= 0;
    };
    static_assert(32 / kClusterGroups == 4, "four clusters per warp step");
    int gnext = -1;
    bool have = cand >= 0 && next_step(gnext);
    if (have) fetch(gnext, cw, cb0, cb1);
    while (have) {
      const int gi = gnext;
      have = next_step(gnext);
      uint32_t nw[6] = {0, 0, 0, 0, 0, 0};
      int nb0 = 0, nb1 = 0;
      if (have) fetch(gnext, nw, nb0, nb1);
      // lane l: its group gi, A and bound
      int A = 0, n = 0;
      const int beg = cb0;
      if (gi >= 0 && gi < p.ngroups) {
        A = (__popc(e & cw[0]) + __popc(o & cw[3])) + 2 * (__popc(e & cw[1]) + __popc(o & cw[4])) +
            4 * (__popc(e & cw[2]) + __popc(o & cw[5]));
        n_bound++;
        if (upper(A, p.C) >= cut) n = cb1 - cb0;
      }
#pragma unroll
      for (int k = 0; k < 6; k++) cw[k] = nw[k];
      cb0 = nb0;
      cb1 = nb1;
      if (!__any_sync(0xFFFFFFFFu, n > 0)) continue;  // no group of this step survives
      // inclusive prefix sum of the surviving members over the lanes
      int incl = n;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += t;
      }
      const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
      for (int base = 0; base < total; base += 32) {
        const int idx = base + lane;
        // the lane L whose range holds idx: the number of lanes with incl <= idx
        int L = 0;
#pragma unroll
        for (int step = 16; step; step >>= 1) {
          const int probe = __shfl_sync(0xFFFFFFFFu, incl, L + step - 1);
          if (probe <= idx) L += step;
        }
        L = min(L, 31);
        const int gA = __shfl_sync(0xFFFFFFFFu, A, L);
        const int gbeg = __shfl_sync(0xFFFFFFFFu, beg, L);
        const int gex = __shfl_sync(0xFFFFFFFFu, incl - n, L);
        if (idx < total) {
          const int m = gbeg + (idx - gex);
          const int orig = __ldg(p.midx + m);
          // B = sum over the H even residues k of #H odd neighbours; the bit tests are uniform
          int B = 0;
#pragma unroll
          for (int k = 0; k < hp::kMaxHalf; k++)
            if ((e >> k) & 1u) B += __popc(o & __ldg(p.mmask + (size_t)k * p.spad + m));
          take(10 * gA + 3 * B, orig);
        }
      }
    }
    const int M = __reduce_max_sync(0xFFFFFFFFu, best);
    const int total = __reduce_add_sync(0xFFFFFFFFu, best == M ? cnt : 0);
    const int f = __reduce_min_sync(0xFFFFFFFFu, best == M ? first : INT_MAX);
    if (GAP) {
      // second-best score over the warp: the best itself when it is tied, else the larger of the
      // lanes' second-best (lanes at M) and best (other lanes) scores; -1 when there is none
      const int x2 = total >= 2 ? M : __reduce_max_sync(0xFFFFFFFFu, best == M ? sec : best);
      int gap = x2 < 0 ? INT_MAX : M - x2;
      if (p.prune) gap = min(gap, p.T);
      if (lane == 0) {
        const int cls = (f >= 0 && f < p.S_dir) ? __ldg(p.conf_class + f) : -1;
        p.phen[q] = gap >= p.T ? cls : -1;
        if (p.aux) p.aux[q] = cls;
        if (p.gap) p.gap[q] = gap;
      }
    } else if (lane == 0) {
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
// counts, so equal vectors form contiguous groups.  The order interleaves the
// counts' bits (the high bit of every residue's count, then the middle bits,
// then the low bits), so that the 32 groups of a cluster have similar counts in
// every residue and the cluster's bound stays tight.
int scan_tables(const hp_structs* cs, DevTables** out) {
  DevTables* dt = nullptr;
  int rc = device_tables(cs, &dt);
  if (rc != HP_OK) return rc;
  hp_structs* s = const_cast<hp_structs*>(cs);
  std::lock_guard<std::mutex> lock(s->mu);
  if (dt->scan_gcnt) {
    *out = dt;
    return HP_OK;
  }
  const int N = s->N, NE = s->NE, W = s->rec_words;
  std::vector<std::vector<uint8_t>> cvec((size_t)s->S_dir, std::vector<uint8_t>(N, 0));
  for (int32_t c = 0; c < s->S_dir; c++)
    for (int k = 0; k < s->C; k++) {
      cvec[c][s->contacts[((size_t)c * s->C + k) * 2]]++;
      cvec[c][s->contacts[((size_t)c * s->C + k) * 2 + 1]]++;
    }
  std::vector<std::vector<uint8_t>> key((size_t)s->S_dir, std::vector<uint8_t>(3 * (size_t)N, 0));
  for (int32_t c = 0; c < s->S_dir; c++)
    for (int b = 2; b >= 0; b--)
      for (int i = 0; i < N; i++) key[c][(size_t)(2 - b) * N + i] = (cvec[c][i] >> b) & 1;
  std::vector<int32_t> order((size_t)s->S_dir);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  std::vector<int32_t> gbeg;
  for (size_t j = 0; j < order.size(); j++)
    if (j == 0 || cvec[order[j]] != cvec[order[j - 1]]) gbeg.push_back((int32_t)j);
  const int ngroups = (int)gbeg.size();
  gbeg.push_back((int32_t)order.size());
  const int gpad = (ngroups + 31) / 32 * 32, spad = (s->S_dir + 31) / 32 * 32;
  const int nclusters = (ngroups + kClusterGroups - 1) / kClusterGroups, cpad = (nclusters + 31) / 32 * 32;
  std::vector<uint32_t> ccnt((size_t)12 * cpad, 0u);
  std::vector<int32_t> cl1(cpad, 0);
  for (int cl = 0; cl < nclusters; cl++) {
    const int g0 = kClusterGroups * cl, g1 = std::min(ngroups, g0 + kClusterGroups);
    std::vector<uint8_t> mn(N, 255), mx(N, 0);
    for (int gi = g0; gi < g1; gi++)
      for (int i = 0; i < N; i++) {
        mn[i] = std::min(mn[i], cvec[order[gbeg[gi]]][i]);
        mx[i] = std::max(mx[i], cvec[order[gbeg[gi]]][i]);
      }
    for (int gi = g0; gi < g1; gi++) {
      int l1 = 0;
      for (int i = 0; i < N; i++) l1 += cvec[order[gbeg[gi]]][i] - mn[i];
      cl1[cl] = std::max(cl1[cl], l1);
    }
    // even residue 2k -> bit k of the even planes, odd residue 2k + 1 -> bit k of the odd planes;
    // planes 0..5 the minimum, 6..11 the largest excess
    for (int i = 0; i < N; i++)
      for (int b = 0; b < 3; b++) {
        const size_t plane = (i & 1) ? 3 + b : b;
        if ((mn[i] >> b) & 1) ccnt[plane * cpad + cl] |= 1u << (i >> 1);
        if (((mx[i] - mn[i]) >> b) & 1) ccnt[(6 + plane) * cpad + cl] |= 1u << (i >> 1);
      }
  }
  std::vector<uint32_t> gcnt((size_t)6 * gpad, 0u), mcnt((size_t)6 * spad, 0u), mmask((size_t)std::max(NE, 1) * spad, 0u);
  std::vector<int32_t> midx(spad, -1);
  for (int gi = 0; gi < ngroups; gi++) {
    const uint32_t* r = s->rec.data() + (size_t)order[gbeg[gi]] * W;  // count planes of any member
    for (int b = 0; b < 3; b++) {
      gcnt[(size_t)b * gpad + gi] = r[NE + 3 + b];
      gcnt[(size_t)(3 + b) * gpad + gi] = r[NE + b];
    }
  }
  for (size_t j = 0; j < order.size(); j++) {
    const uint32_t* r = s->rec.data() + (size_t)order[j] * W;
    for (int k = 0; k < NE; k++) mmask[(size_t)k * spad + j] = r[k];
    for (int b = 0; b < 3; b++) {
      mcnt[(size_t)b * spad + j] = r[NE + 3 + b];
      mcnt[(size_t)(3 + b) * spad + j] = r[NE + b];
    }
    midx[j] = order[j];
  }
  cudaError_t e = cudaMalloc(&dt->scan_gcnt, gcnt.size() * 4);
  if (e == cudaSuccess) e = cudaMalloc(&dt->scan_ccnt, ccnt.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(dt->scan_ccnt, ccnt.data(), ccnt.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&dt->scan_cl1, cl1.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(dt->scan_cl1, cl1.data(), cl1.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&dt->scan_gbeg, gbeg.size() * 4);
  if (e == cudaSuccess) e = cudaMalloc(&dt->scan_mcnt, mcnt.size() * 4);
  if (e == cudaSuccess) e = cudaMalloc(&dt->scan_mmask, mmask.size() * 4);
  if (e == cudaSuccess) e = cudaMalloc(&dt->scan_midx, midx.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(dt->scan_gcnt, gcnt.data(), gcnt.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dt->scan_gbeg, gbeg.data(), gbeg.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dt->scan_mcnt, mcnt.data(), mcnt.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dt->scan_mmask, mmask.data(), mmask.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dt->scan_midx, midx.data(), midx.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dt->scan_gcnt);
    cudaFree(dt->scan_ccnt);
    cudaFree(dt->scan_cl1);
    cudaFree(dt->scan_gbeg);
    cudaFree(dt->scan_mcnt);
    cudaFree(dt->scan_mmask);
    cudaFree(dt->scan_midx);
    dt->scan_mcnt = nullptr;
    dt->scan_gcnt = nullptr;
    dt->scan_ccnt = nullptr;
    dt->scan_cl1 = nullptr;
    dt->scan_gbeg = nullptr;
    dt->scan_mmask = nullptr;
    dt->scan_midx = nullptr;
    return cuda_fail(e, "per-sequence scan tables");
  }
  dt->scan_ngroups = ngroups;
  dt->scan_gpad = gpad;
  dt->scan_cpad = cpad;
  dt->scan_spad = spad;
  *out = dt;
  return HP_OK;
}

}  // namespace hp

namespace {

constexpr int kMaxGapThreshold = 1 << 20;

// One launch of the scan over n ids.
int launch_scan(const hp_structs* s, const uint64_t* d_ids, int64_t n, const int32_t* d_cand,
                int32_t k, int32_t T, bool gap_variant, int32_t* d_phen, int32_t* d_aux, int32_t* d_gap,
                uint64_t* d_counters, cudaStream_t stream) {
  hp::DevTables* dt = nullptr;
  int rc = hp::scan_tables(s, &dt);
  if (rc != HP_OK) return rc;
  ScanParams p;
  p.gcnt = dt->scan_gcnt;
  p.ccnt = dt->scan_ccnt;
  p.cl1 = dt->scan_cl1;
  p.nclusters = (dt->scan_ngroups + kClusterGroups - 1) / kClusterGroups;
  p.cpad = dt->scan_cpad;
  p.gbeg = dt->scan_gbeg;
  p.mcnt = dt->scan_mcnt;
  p.mmask = dt->scan_mmask;
  p.midx = dt->scan_midx;
  p.orig_rec = dt->rec;
  p.conf_class = dt->conf_class;
  p.ids = reinterpret_cast<const unsigned long long*>(d_ids);
  p.cand = d_cand;
  p.phen = d_phen;
  p.aux = d_aux;
  p.gap = d_gap;
  p.counters = reinterpret_cast<unsigned long long*>(d_counters);
  p.n = n;
  p.k = k;
  p.rec_words = s->rec_words;
  p.NE = s->NE;
  p.C = s->C;
  p.S_dir = s->S_dir;
  p.ngroups = dt->scan_ngroups;
  p.gpad = dt->scan_gpad;
  p.spad = dt->scan_spad;
  p.prune = d_cand != nullptr;
  p.T = T;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (n + kScanWarps - 1) / kScanWarps;
  blocks = std::min<long long>(blocks, (long long)sms * 8);
  if (gap_variant)
    seq_scan_kernel<true><<<(unsigned)blocks, 32 * kScanWarps, 0, stream>>>(p);
  else
    seq_scan_kernel<false><<<(unsigned)blocks, 32 * kScanWarps, 0, stream>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hp::cuda_fail(e, "per-sequence scan: launch");
  return HP_OK;
}

}  // namespace

extern "C" int hp_sequence_scan_gap(const hp_structs* s, const uint64_t* d_ids, int64_t n, const int32_t* d_cand,
                                    int32_t k, int32_t gap_threshold, int32_t* d_phen, int32_t* d_aux,
                                    int32_t* d_gap, uint64_t* d_counters, void* stream) {
  if (!s || !d_ids || !d_phen) return hp::fail(HP_EINVAL, "hp_sequence_scan: NULL argument");
  if (n < 0 || k < 0 || (d_cand && k == 0)) return hp::fail(HP_EINVAL, "hp_sequence_scan: bad sizes");
  if (gap_threshold < 1 || gap_threshold > kMaxGapThreshold)
    return hp::fail(HP_EINVAL, "hp_sequence_scan: gap_threshold must be in [1, 2^20]");
  if (s->N > 2 * hp::kMaxHalf) return hp::fail(HP_EUNSUPPORTED, "hp_sequence_scan: N > 40");
  if (n == 0) return HP_OK;
  const bool gap_variant = gap_threshold != 1 || d_gap != nullptr;
  return launch_scan(s, d_ids, n, d_cand, k, gap_threshold, gap_variant, d_phen, d_aux, d_gap, d_counters,
                     (cudaStream_t)stream);
}

extern "C" int hp_sequence_scan(const hp_structs* s, const uint64_t* d_ids, int64_t n, const int32_t* d_cand,
                                int32_t k, int32_t* d_phen, int32_t* d_aux, uint64_t* d_counters, void* stream) {
  return hp_sequence_scan_gap(s, d_ids, n, d_cand, k, 1, d_phen, d_aux, nullptr, d_counters, stream);
}
