// The full matrix of Eq. 2 numerators (Section 2.3 of arXiv 2008.05612): for every ordered pair of
// phenotypes (q, p), the number of single flips from a genotype of q to a genotype of p,
//   M[q][p] = #{(g, i) : P(g) = q, P(g xor 2^i) = p},  phi_pq = M[q][p] / (N N_q),
// with index S standing for the deleterious phenotype -1.  The matrix is sparse (a phenotype's
// neighbours are few: 0.86% of the 3x3x3 phenotypes touch the top fold, Section 3.2), so it is
// returned in compressed rows with columns ascending.
//
// Where the counts come from.  The diagonal M[p][p] and the -1 column M[p][S] are the robustness
// numerators (the same tile pass as hp_robustness); flips are symmetric (g -> h is a flip iff
// h -> g is), so the -1 row is the -1 column transposed, M[S][p] = M[p][S].  Only the flips between
// two different non-deleterious phenotypes (4% of the 3x3x3 neighbours) go through a hash table
// keyed by (q, p).  The entries are then sorted by (row, column) with a bitonic sort and the row
// offsets found by binary search.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "hp_internal.h"

namespace {

constexpr unsigned kErrRange = 4u;   // a map entry outside [-1, S)
constexpr unsigned kErrFull = 16u;   // the hash table is full
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr int kTileBits = 14;        // 2^14 ids of the map per CTA (flips of the low bits in shared memory)
constexpr int kThreads = 512;

__device__ __forceinline__ uint32_t slot_of(uint32_t key, int log2cap) { return (key * 0x9E3779B1u) >> (32 - log2cap); }

// Add 1 to the count of key (q << 16 | p) in the open-addressing table (linear probing, bounded).
__device__ __forceinline__ void hash_add(uint32_t* keys, unsigned long long* counts, int log2cap, uint32_t key,
                                         unsigned* err) {
  const uint32_t mask = (1u << log2cap) - 1u;
  uint32_t s = slot_of(key, log2cap);
  for (uint32_t probe = 0; probe <= mask; probe++, s = (s + 1) & mask) {
    uint32_t k = keys[s];
    if (k == kEmpty) {
      k = atomicCAS(keys + s, kEmpty, key);
      if (k == kEmpty) k = key;
    }
    if (k == key) {
      atomicAdd(counts + s, 1ull);
      return;
    }
  }
  atomicOr(err, kErrFull);
}

// Flips between two different non-deleterious phenotypes, one CTA per 2^kTileBits ids (low-bit
// partners from shared memory, high-bit partners from global memory).
__global__ void __launch_bounds__(kThreads) phi_offdiag(const int32_t* __restrict__ phen, int N, int S, uint32_t* keys,
                                                        unsigned long long* counts, int log2cap, unsigned* err) {
  extern __shared__ int32_t tile[];
  const int k = min(N, kTileBits);
  const unsigned long long tsize = 1ull << k;
  const unsigned long long g0 = (unsigned long long)blockIdx.x << k;
  for (unsigned long long j = threadIdx.x; j < tsize; j += blockDim.x) tile[j] = __ldcs(phen + g0 + j);
  __syncthreads();
  for (unsigned long long j = threadIdx.x; j < tsize; j += blockDim.x) {
    const int32_t q = tile[j];
    if (q < 0 || q >= S) {
      if (q < -1 || q >= S) atomicOr(err, kErrRange);
      continue;
    }
    const unsigned long long g = g0 + j;
    for (int i = 0; i < N; i++) {
      const int32_t p = i < k ? tile[j ^ (1ull << i)] : __ldg(phen + (g ^ (1ull << i)));
      if (p >= 0 && p != q && p < S) hash_add(keys, counts, log2cap, ((uint32_t)q << 16) | (uint32_t)p, err);
    }
  }
}

// Store entry `at` unless it lies beyond the output's `limit` entries (then it is only counted).
__device__ __forceinline__ void put(uint32_t* out_key, unsigned long long* out_cnt, unsigned long long limit,
                                    unsigned long long at, uint32_t key, unsigned long long cnt) {
  if (at < limit) {
    out_key[at] = key;
    out_cnt[at] = cnt;
  }
}

// The diagonal (neutral[p]), the -1 column and row (to_del[p]) and the -1/-1 entry, appended after
// the *base compacted hash entries (slots from the cursor).
__global__ void phi_structured(const unsigned long long* __restrict__ neutral, const unsigned long long* __restrict__ to_del,
                               int S, const unsigned long long* __restrict__ base, uint32_t* out_key,
                               unsigned long long* out_cnt, unsigned long long limit, unsigned long long* cursor) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > S) return;
  const unsigned long long b = *base;
  if (p < S) {
    if (neutral[p]) put(out_key, out_cnt, limit, b + atomicAdd(cursor, 1ull), ((uint32_t)p << 16) | (uint32_t)p, neutral[p]);
    if (to_del[p]) {
      const unsigned long long at = b + atomicAdd(cursor, 2ull);
      put(out_key, out_cnt, limit, at, ((uint32_t)p << 16) | (uint32_t)S, to_del[p]);
      put(out_key, out_cnt, limit, at + 1, ((uint32_t)S << 16) | (uint32_t)p, to_del[p]);
    }
  } else if (neutral[S]) {
    put(out_key, out_cnt, limit, b + atomicAdd(cursor, 1ull), ((uint32_t)S << 16) | (uint32_t)S, neutral[S]);
  }
}

// Compact the occupied hash slots to the front of (out_key, out_cnt); *n counts them.
__global__ void phi_compact(const uint32_t* __restrict__ keys, const unsigned long long* __restrict__ counts,
                            unsigned long long hcap, uint32_t* out_key, unsigned long long* out_cnt,
                            unsigned long long limit, unsigned long long* n) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < hcap; s += stride) {
    const uint32_t k = keys[s];
    if (k == kEmpty) continue;
    put(out_key, out_cnt, limit, atomicAdd(n, 1ull), k, counts[s]);
  }
}

// One compare-exchange step of a bitonic sort over `len` (a power of two) keys with their counts.
__global__ void bitonic_step(uint32_t* key, unsigned long long* cnt, unsigned long long len, unsigned long long j,
                             unsigned long long k) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
    const unsigned long long l = i ^ j;
    if (l <= i) continue;
    const bool up = (i & k) == 0;
    const uint32_t a = key[i], b = key[l];
    if ((a > b) == up) {
      key[i] = b;
      key[l] = a;
      const unsigned long long t = cnt[i];
      cnt[i] = cnt[l];
      cnt[l] = t;
    }
  }
}

// Row offsets: row_ptr[q] = first entry with row >= q (binary search over the sorted keys); the
// columns and counts are copied out.
__global__ void phi_rows(const uint32_t* __restrict__ key, unsigned long long nnz, int S, uint64_t* row_ptr) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > S + 1) return;
  const uint32_t want = (uint32_t)q << 16;
  unsigned long long lo = 0, hi = nnz;
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) / 2;
    if (key[mid] < want) lo = mid + 1;
    else hi = mid;
  }
  row_ptr[q] = lo;
}

__global__ void phi_columns(const uint32_t* __restrict__ key, const unsigned long long* __restrict__ cnt,
                            unsigned long long nnz, int32_t* col, uint64_t* count) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride) {
    col[i] = (int32_t)(key[i] & 0xFFFFu);
    count[i] = cnt[i];
  }
}

int sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace

extern "C" int hp_phi_matrix(const int32_t* d_phen, int32_t N, int32_t S, uint64_t cap, uint64_t* d_row_ptr,
                             int32_t* d_col, uint64_t* d_count, uint64_t* h_nnz, void* stream) {
  if (!d_phen || !d_row_ptr || !d_col || !d_count || !h_nnz) return hp::fail(HP_EINVAL, "hp_phi_matrix: NULL pointer");
  if (N < 1 || N > 40) return hp::fail(HP_EINVAL, "hp_phi_matrix: N must be in [1, 40]");
  if (S < 1 || S >= 0xFFFF) return hp::fail(HP_EINVAL, "hp_phi_matrix: S must be in [1, 65534]");
  if (cap < 1 || cap > (1ull << 30)) return hp::fail(HP_EINVAL, "hp_phi_matrix: cap must be in [1, 2^30]");
  cudaStream_t st = (cudaStream_t)stream;
  *h_nnz = 0;
  // hash table: twice the off-diagonal capacity, a power of two (at least 2^10)
  int log2cap = 10;
  while ((1ull << log2cap) < 2 * cap && log2cap < 31) log2cap++;
  const unsigned long long hcap = 1ull << log2cap;
  unsigned long long slen = 1;  // sort buffer: the output's capacity, a power of two
  while (slen < cap) slen <<= 1;
  // scratch: [err 8][n 8][cursor 8][negcount 8][neutral (S+1)][to_del (S+1)] | keys | counts | sort keys | sort counts
  const size_t head = 32 + 16ull * (size_t)(S + 1);
  const size_t bytes = head + hcap * 4 + hcap * 8 + slen * 4 + slen * 8;
  char* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), bytes, st);
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_phi_matrix: cudaMallocAsync");
  unsigned* err = reinterpret_cast<unsigned*>(scratch);
  unsigned long long* n = reinterpret_cast<unsigned long long*>(scratch + 8);
  unsigned long long* cursor = reinterpret_cast<unsigned long long*>(scratch + 16);
  unsigned long long* negcount = reinterpret_cast<unsigned long long*>(scratch + 24);
  unsigned long long* neutral = reinterpret_cast<unsigned long long*>(scratch + 32);
  unsigned long long* to_del = neutral + (S + 1);
  uint32_t* keys = reinterpret_cast<uint32_t*>(scratch + head);
  unsigned long long* counts = reinterpret_cast<unsigned long long*>(scratch + head + hcap * 4);
  uint32_t* skey = reinterpret_cast<uint32_t*>(scratch + head + hcap * 12);
  unsigned long long* scnt = reinterpret_cast<unsigned long long*>(scratch + head + hcap * 12 + slen * 4);
  int rc = HP_OK;
  e = cudaMemsetAsync(scratch, 0, head, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(keys, 0xFF, hcap * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, hcap * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(skey, 0xFF, slen * 4, st);
  if (e == cudaSuccess) e = hp::launch_robustness(d_phen, N, S, neutral, to_del, negcount, err, st);
  const int k = std::min((int)N, kTileBits);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(phi_offdiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(4 << k));
  if (e == cudaSuccess) {
    phi_offdiag<<<(unsigned)(1ull << (N - k)), kThreads, 4 << k, st>>>(d_phen, N, S, keys, counts, log2cap, err);
    const unsigned grid = (unsigned)std::min<unsigned long long>((hcap + 255) / 256, (unsigned long long)sms() * 16);
    phi_compact<<<grid, 256, 0, st>>>(keys, counts, hcap, skey, scnt, cap, n);
    phi_structured<<<(S + 1 + 255) / 256, 256, 0, st>>>(neutral, to_del, S, n, skey, scnt, cap, cursor);
    e = cudaGetLastError();
  }
  // read back the error word and the entry counts before sorting (the sort length depends on them)
  unsigned long long hn[2] = {0, 0};
  unsigned herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hn, n, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_phi_matrix: counting");
  const unsigned long long nnz = hn[0] + hn[1];
  if (rc == HP_OK && (herr & kErrRange)) rc = hp::fail(HP_EINVAL, "hp_phi_matrix: map entry outside [-1, S)");
  if (rc == HP_OK && ((herr & kErrFull) || nnz > cap)) {
    *h_nnz = (herr & kErrFull) ? 0 : nnz;
    rc = hp::fail(HP_ENOMEM, "hp_phi_matrix: the matrix has more than cap = " + std::to_string(cap) +
                                 " nonzero entries; call again with cap >= *h_nnz (0: unknown, at least 2 x cap)");
  }
  if (rc == HP_OK) {
    unsigned long long len = 1;
    while (len < nnz) len <<= 1;
    const unsigned grid = (unsigned)std::min<unsigned long long>((len + 255) / 256, (unsigned long long)sms() * 16);
    for (unsigned long long kk = 2; kk <= len; kk <<= 1)
      for (unsigned long long j = kk >> 1; j > 0; j >>= 1) bitonic_step<<<grid, 256, 0, st>>>(skey, scnt, len, j, kk);
    phi_rows<<<(S + 2 + 255) / 256, 256, 0, st>>>(skey, nnz, S, d_row_ptr);
    if (nnz)
      phi_columns<<<(unsigned)std::min<unsigned long long>((nnz + 255) / 256, (unsigned long long)sms() * 16), 256, 0, st>>>(
          skey, scnt, nnz, d_col, d_count);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_phi_matrix: sort");
    else *h_nnz = nnz;
  }
  cudaFreeAsync(scratch, st);
  return rc;
}
