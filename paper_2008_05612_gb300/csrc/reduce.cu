// Reductions of a phenotype map (Section 2.3 of arXiv 2008.05612):
// designability, the Eq. 2 numerators behind robustness and phi_del, and the
// neutral networks (connected components of same-phenotype single flips).
// All three are HBM-bound passes over the int32 map.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "hp_internal.h"

namespace {

constexpr unsigned kErrRange = 4u;     // a map entry outside [-1, S)
constexpr unsigned kErrUnion = 8u;     // union retries exhausted
constexpr int kHistThreads = 1024;
constexpr int kRobTileBits = 13;       // 2^13 ids (32 KB) of the map per block, two blocks per CTA
constexpr int kRobMaxPassBits = 8;     // high bits per later pass (a block keeps >= 32 contiguous ids)
constexpr int kRobThreads = 512;
constexpr int kRobReplicas = 16;       // copies of each phenotype's two counters (spreads hot-phenotype atomics)

// ---------------------------------------------------------------- designability

// Privatised histogram in shared memory, one partial row per CTA.  Entry -1 is
// by far the most common (95% of 3x3x3 genotypes), so it is counted in a
// register and added once per warp.
__global__ void __launch_bounds__(kHistThreads) hist_partial(const int32_t* __restrict__ phen, unsigned long long count,
                                                             int S, unsigned* __restrict__ partial,
                                                             unsigned* __restrict__ err, int vec4) {
  extern __shared__ unsigned bins[];
  for (int b = threadIdx.x; b <= S; b += blockDim.x) bins[b] = 0u;
  __syncthreads();
  unsigned neg = 0, bad = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  auto take = [&](int32_t p) {
    if (p < 0) {
      if (p == -1) neg++; else bad = 1;
    } else if (p < S) {
      atomicAdd(&bins[p], 1u);
    } else {
      bad = 1;
    }
  };
  unsigned long long done = 0;
  if (vec4) {
    const int4* v = reinterpret_cast<const int4*>(phen);
    const unsigned long long nv = count / 4;
    // four 16-byte loads of a thread in flight together, then their ids binned
    unsigned long long k = t0;
    for (; k + 3 * stride < nv; k += 4 * stride) {
      int4 q[4];
#pragma unroll
      for (int u = 0; u < 4; u++) q[u] = __ldcs(v + k + u * stride);
#pragma unroll
      for (int u = 0; u < 4; u++) {
        take(q[u].x); take(q[u].y); take(q[u].z); take(q[u].w);
      }
    }
    for (; k < nv; k += stride) {
      const int4 q = __ldcs(v + k);
      take(q.x); take(q.y); take(q.z); take(q.w);
    }
    done = nv * 4;
  }
  for (unsigned long long k = done + t0; k < count; k += stride) take(__ldcs(phen + k));
  for (int off = 16; off; off >>= 1) neg += __shfl_xor_sync(0xFFFFFFFFu, neg, off);
  if ((threadIdx.x & 31) == 0 && neg) atomicAdd(&bins[S], neg);
  if (bad) atomicOr(err, kErrRange);
  __syncthreads();
  unsigned* row = partial + (size_t)blockIdx.x * (S + 1);
  for (int b = threadIdx.x; b <= S; b += blockDim.x) row[b] = bins[b];
}

// hist[b] = (accumulate ? hist[b] : 0) + the column sum of the partial rows
__global__ void hist_sum(const unsigned* __restrict__ partial, int rows, int S, unsigned long long* __restrict__ hist,
                         int accumulate) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > S) return;
  unsigned long long s = accumulate ? hist[b] : 0ull;
  for (int r = 0; r < rows; r++) s += partial[(size_t)r * (S + 1) + b];
  hist[b] = s;
}

// Ids one partial row may count before its uint32 bins could wrap (a row counts about
// count / rows ids, most of them into one bin): ranges beyond rows x this are split into passes.
constexpr unsigned long long kHistIdsPerRow = 1ull << 31;

// hist_partial + hist_sum over [0, count) in passes of at most rows x kHistIdsPerRow ids (a
// multiple of 4, so every pass keeps the 16-byte alignment of d_phen), the later passes adding to
// d_hist.
cudaError_t launch_hist(const int32_t* d_phen, unsigned long long count, int S, unsigned* partial, int rows,
                        unsigned* err, uint64_t* d_hist, size_t bins_bytes, cudaStream_t st) {
  const int vec4 = ((uintptr_t)d_phen % 16) == 0;
  const unsigned long long pass = (unsigned long long)rows * kHistIdsPerRow;
  for (unsigned long long off = 0; off < count; off += pass) {
    const unsigned long long n = std::min(pass, count - off);
    hist_partial<<<rows, kHistThreads, bins_bytes, st>>>(d_phen + off, n, S, partial, err, vec4);
    hist_sum<<<(S + 1 + 255) / 256, 256, 0, st>>>(partial, rows, S, reinterpret_cast<unsigned long long*>(d_hist),
                                                 off > 0);
  }
  return cudaGetLastError();
}

// fallback for phenotype counts too large for one shared-memory histogram
__global__ void hist_global(const int32_t* __restrict__ phen, unsigned long long count, int S,
                            unsigned long long* __restrict__ hist, unsigned* __restrict__ err) {
  unsigned neg = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
    const int32_t p = phen[k];
    if (p == -1) neg++;
    else if (p >= 0 && p < S) atomicAdd(&hist[p], 1ull);
    else atomicOr(err, kErrRange);
  }
  for (int off = 16; off; off >>= 1) neg += __shfl_xor_sync(0xFFFFFFFFu, neg, off);
  if ((threadIdx.x & 31) == 0 && neg) atomicAdd(&hist[S], (unsigned long long)neg);
}

// ---------------------------------------------------------------- robustness

// Eq. 2 numerators in passes over the map, each reading it once.  A block is 2^kRobTileBits ids
// in shared memory: 2^c consecutive ids times every combination of the pass's h bits
// (c + h = kRobTileBits), the other bits of the id fixed by the block index.  The first pass
// takes 2^13 consecutive ids and counts the flips of bits 0..12; each later pass counts the flips
// of its own h bits, so every flip of every genotype is counted once, from shared memory, with
// the map read 1 + ceil((N - 13) / 8) times instead of once per high bit.  Only genotypes with
// P(g) >= 0 examine their flips; the -1 row follows from the edge identity
// sum_{P(g)=-1} #{i: P(g^2^i) = -1} = N N_{-1} - sum_{p>=0} to_del[p].
// A CTA walks blocks with the next block's asynchronous copy in flight; the block's genotypes
// that fold are listed first, then examined one per lane.  The counts go to replica blockIdx % R of each phenotype's counters
// (neutral[r S + p], to_del[r S + p]), so that the atomics of a very designable phenotype are
// spread over R addresses; robustness_gather adds the replicas up.
struct RobPass {
  int c, h;                   // contiguous low bits of a block; pass bits
  int pos[kRobMaxPassBits];   // positions of the pass bits (all >= c)
  int nrest;                  // the remaining id bits, filled from the block index (low bit first)
  int rest[64];
  int first;                  // first pass: counts the contiguous bits' flips, checks ranges, counts -1
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

__global__ void __launch_bounds__(kRobThreads) robustness_pass(const int32_t* __restrict__ phen, int S, const RobPass P,
                                                               unsigned long long nblocks, int replicas,
                                                               unsigned long long* __restrict__ neutral_rep,
                                                               unsigned long long* __restrict__ to_del_rep,
                                                               unsigned long long* __restrict__ negcount,
                                                               unsigned* __restrict__ err) {
  extern __shared__ int32_t tiles[];  // two blocks, then the list of a block's genotypes that fold
  __shared__ unsigned long long hoff[1 << kRobMaxPassBits];
  __shared__ unsigned nlist;
  constexpr int kIds = 1 << kRobTileBits;
  uint16_t* list = reinterpret_cast<uint16_t*>(tiles + 2 * kIds);
  static_assert(kRobTileBits <= 16, "list entries are 16-bit local indices");
  for (int i = threadIdx.x; i < (1 << P.h); i += blockDim.x) {
    unsigned long long off = 0;
    for (int t = 0; t < P.h; t++)
      if ((i >> t) & 1) off |= 1ull << P.pos[t];
    hoff[i] = off;
  }
  __syncthreads();
  const int c = P.c;
  const unsigned cmask = (1u << c) - 1u, ids = 1u << (c + P.h);  // ids < kIds only when N < kRobTileBits
  const bool vec = reinterpret_cast<uintptr_t>(phen) % 16 == 0 && c >= 2 && ids == (unsigned)kIds;
  auto block_base = [&](unsigned long long b) {
    unsigned long long base = 0;
    for (int t = 0; t < P.nrest; t++)
      if ((b >> t) & 1ull) base |= 1ull << P.rest[t];
    return base;
  };
  // block b into slot: 16-byte asynchronous copies (four ids never straddle two runs when c >= 2)
  constexpr int kLoads = kIds / (4 * kRobThreads);
  auto issue = [&](unsigned long long b, int slot) {
    const unsigned long long base = block_base(b);
    int32_t* t = tiles + slot * kIds;
#pragma unroll
    for (int k = 0; k < kLoads; k++) {
      const unsigned j = 4 * (threadIdx.x + k * kRobThreads);
      cp_async16(t + j, phen + base + hoff[j >> c] + (j & cmask));
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // counted flips: local bits 0..c-1 in the first pass, c..c+h-1 in the others
  const int nbits = P.first ? c : P.h, bit0 = P.first ? 0 : c;
  const int lane = threadIdx.x & 31;
  unsigned long long* __restrict__ neutral = neutral_rep + (size_t)(blockIdx.x % replicas) * S;
  unsigned long long* __restrict__ to_del = to_del_rep + (size_t)(blockIdx.x % replicas) * S;
  unsigned neg = 0;
  unsigned long long b = blockIdx.x;
  if (vec && b < nblocks) issue(b, 0);
  for (int it = 0; b < nblocks; b += gridDim.x, it++) {
    int32_t* tile = tiles + (it & 1) * kIds;
    if (threadIdx.x == 0) nlist = 0;  // ordered before phase 1 by the barrier after the load
    const unsigned long long nb = b + gridDim.x;
    if (vec) {
      if (nb < nblocks) {
        issue(nb, (it + 1) & 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
    } else {
      const unsigned long long base = block_base(b);
      for (unsigned j = threadIdx.x; j < ids; j += blockDim.x) tile[j] = __ldcs(phen + base + hoff[j >> c] + (j & cmask));
    }
    __syncthreads();
    // phase 1: the block's genotypes that fold, listed (local indices) in shared memory; whole
    // warps, four ids per lane (one 16-byte read), branch-free; the first pass also counts -1 and
    // checks the ranges
    for (unsigned j0 = 4 * (threadIdx.x - lane); j0 < ids; j0 += 4 * blockDim.x) {
      const unsigned j = j0 + 4 * lane;
      int4 v4 = make_int4(-1, -1, -1, -1);
      if (j + 3 < ids) {
        v4 = *reinterpret_cast<const int4*>(tile + j);
      } else if (j < ids) {  // blocks of fewer than four ids (maps of N < 2)
        v4.x = tile[j];
        if (j + 1 < ids) v4.y = tile[j + 1];
        if (j + 2 < ids) v4.z = tile[j + 2];
      }
      const int32_t e[4] = {v4.x, v4.y, v4.z, v4.w};
      unsigned flags = 0;
#pragma unroll
      for (int k = 0; k < 4; k++) flags |= (unsigned)((unsigned)e[k] < (unsigned)S) << k;
      if (P.first) {
        const unsigned valid = j < ids ? min(4u, ids - j) : 0u;
#pragma unroll
        for (int k = 0; k < 4; k++) {
          neg += (unsigned)(k < (int)valid && e[k] == -1);
          if (k < (int)valid && (e[k] < -1 || e[k] >= S)) atomicOr(err, kErrRange);
        }
      }
      // this lane's place in the list: the folding ids of the lanes below it (cnt <= 4, three bits)
      const unsigned cnt = __popc(flags);
      const uint32_t lt = (1u << lane) - 1u;
      const uint32_t b0 = __ballot_sync(0xFFFFFFFFu, cnt & 1u), b1 = __ballot_sync(0xFFFFFFFFu, cnt & 2u),
                     b2 = __ballot_sync(0xFFFFFFFFu, cnt & 4u);
      const unsigned below = __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt);
      const unsigned tot = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
      unsigned at = 0;
      if (lane == 0 && tot) at = atomicAdd(&nlist, tot);
      at = __shfl_sync(0xFFFFFFFFu, at, 0) + below;
#pragma unroll
      for (int k = 0; k < 4; k++)
        if (flags & (1u << k)) list[at++] = (uint16_t)(j + k);
    }
    __syncthreads();
    // phase 2: one listed genotype per lane, its counted flips in turn
    {
      const unsigned n = nlist;
      for (unsigned f = threadIdx.x; f < n; f += blockDim.x) {
        const unsigned idx = list[f];
        const int32_t p = tile[idx];
        unsigned nn = 0, nd = 0;
        for (int t = 0; t < nbits; t++) {
          const int32_t q = tile[idx ^ (1u << (bit0 + t))];
          nn += q == p;
          nd += q < 0;
        }
        if (nn) atomicAdd(&neutral[p], (unsigned long long)nn);
        if (nd) atomicAdd(&to_del[p], (unsigned long long)nd);
      }
    }
    __syncthreads();  // the slot is refilled by the copy issued in the next iteration but one
  }
  if (P.first) {
    for (int off = 16; off; off >>= 1) neg += __shfl_xor_sync(0xFFFFFFFFu, neg, off);
    if (lane == 0 && neg) atomicAdd(negcount, (unsigned long long)neg);
  }
}

__global__ void robustness_gather(const unsigned long long* __restrict__ rep, int replicas, int S,
                                  unsigned long long* __restrict__ neutral, unsigned long long* __restrict__ to_del) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= S) return;
  unsigned long long a = 0, d = 0;
  for (int r = 0; r < replicas; r++) {
    a += rep[(size_t)r * S + p];
    d += rep[(size_t)(replicas + r) * S + p];
  }
  neutral[p] = a;
  to_del[p] = d;
}

__global__ void robustness_finish(int N, int S, unsigned long long* __restrict__ neutral,
                                  unsigned long long* __restrict__ to_del, const unsigned long long* __restrict__ negcount) {
  __shared__ unsigned long long part[32];
  unsigned long long s = 0;
  for (int p = threadIdx.x; p < S; p += blockDim.x) s += to_del[p];
  for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
    const unsigned long long v = (unsigned long long)N * negcount[0] - t;
    neutral[S] = v;
    to_del[S] = v;
  }
}

// ---------------------------------------------------------------- components

__global__ void cc_init(const int32_t* __restrict__ phen, unsigned long long total, int S, int32_t* __restrict__ label,
                        unsigned* __restrict__ err) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    const int32_t p = phen[g];
    if (p < -1 || p >= S) atomicOr(err, kErrRange);
    label[g] = (p >= 0 && p < S) ? (int32_t)g : -1;
  }
}

// Root of x: parents always have smaller ids, so the walk terminates.
__device__ __forceinline__ int32_t cc_root(const int32_t* label, int32_t x) {
  int32_t par = __ldcg(label + x);
  while (par != x) {
    x = par;
    par = __ldcg(label + x);
  }
  return x;
}

// The same with path halving, while components are being joined: each visited id is pointed at
// its grandparent (an ancestor with a smaller id, so concurrent finds and hooks stay correct;
// hooks only change roots, which are never rewritten).  Not for the final compression, where a
// late halving write could replace an id's final root by a non-root ancestor.
__device__ __forceinline__ int32_t cc_find(int32_t* label, int32_t x) {
  for (;;) {
    const int32_t q = __ldcg(label + x);
    if (q == x) return x;
    const int32_t g = __ldcg(label + q);
    if (g == q) return q;
    __stcg(label + x, g);
    x = g;
  }
}

// Lock-free union of the components of a and b: hook the larger root under the smaller one with
// a CAS and retry from the value the CAS saw.  Every failed CAS means another thread linked that
// root, so the loop makes progress; it is bounded all the same (false if it gives up).
__device__ __forceinline__ bool cc_union(int32_t* label, int32_t a, int32_t b) {
  for (int tries = 0; tries < (1 << 24); tries++) {
    const int32_t ra = cc_find(label, a), rb = cc_find(label, b);
    if (ra == rb) return true;
    const int32_t lo = min(ra, rb), hi = max(ra, rb);
    const int32_t seen = atomicCAS(label + hi, hi, lo);
    if (seen == hi) return true;
    a = lo;
    b = seen;
  }
  return false;
}

// One warp per 32 consecutive ids: the (id, flipped bit) pairs of its non-deleterious ids are
// spread over the lanes (about 1.5 such ids per 32 in 3x3x3), so the partner reads and unions of
// different pairs are in flight together instead of one lane walking all N bits.
__global__ void cc_hook(const int32_t* __restrict__ phen, int N, int32_t* label, unsigned* __restrict__ err) {
  const unsigned long long total = 1ull << N;
  const int lane = threadIdx.x & 31;
  const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  for (unsigned long long base = ((unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
       base < total; base += warps * 32) {
    const unsigned long long g = base + lane;
    const bool fold = g < total && __ldcg(label + g) >= 0;  // deleterious ids carry label -1
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, fold);
    const int npairs = __popc(bal) * N;
    for (int k = lane; k < npairs; k += 32) {
      const int src = __fns(bal, 0, k / N + 1), i = k % N;
      const unsigned long long gs = base + src, h = gs ^ (1ull << i);
      if (h < gs) continue;  // each pair once, from its smaller id
      if (__ldg(phen + h) != __ldg(phen + gs)) continue;
      if (!cc_union(label, (int32_t)gs, (int32_t)h)) atomicOr(err, kErrUnion);
    }
  }
}

__global__ void cc_finish(const int32_t* __restrict__ phen, unsigned long long total, int32_t* label,
                          unsigned long long* __restrict__ ncomp) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    const int32_t l = label[g];
    if (l < 0) continue;
    const int32_t r = cc_root(label, (int32_t)g);
    label[g] = r;
    if (r == (int32_t)g) atomicAdd(&ncomp[phen[g]], 1ull);
  }
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Read the error word back (synchronising the stream) and free it.
int finish_with_err(unsigned* err, cudaStream_t st, const char* what, int rc) {
  unsigned herr = 0;
  if (rc == HP_OK) {
    cudaError_t e = cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = hp::cuda_fail(e, what);
  }
  cudaFreeAsync(err, st);
  if (rc == HP_OK && (herr & kErrRange)) rc = hp::fail(HP_EINVAL, std::string(what) + ": map entry outside [-1, S)");
  if (rc == HP_OK && (herr & kErrUnion)) rc = hp::fail(HP_ETIMEOUT, std::string(what) + ": union retries exhausted");
  return rc;
}

}  // namespace

extern "C" int hp_designability(const int32_t* d_phen, uint64_t count, int32_t S, uint64_t* d_hist, void* stream) {
  if (!d_phen || !d_hist) return hp::fail(HP_EINVAL, "hp_designability: NULL pointer");
  if (S < 1) return hp::fail(HP_EINVAL, "hp_designability: S must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* err = nullptr;
  cudaError_t e = cudaMallocAsync(&err, sizeof(unsigned), st);
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_designability: cudaMallocAsync");
  cudaMemsetAsync(err, 0, sizeof(unsigned), st);
  int rc = HP_OK;
  const size_t bins_bytes = (size_t)(S + 1) * sizeof(unsigned);
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (count == 0) {
    e = cudaMemsetAsync(d_hist, 0, sizeof(uint64_t) * (size_t)(S + 1), st);
    if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_designability: memset");
  } else if (bins_bytes <= (size_t)max_smem) {
    int rows = sm_count();
    const unsigned long long need = (count + kHistThreads * 4ull - 1) / (kHistThreads * 4ull);
    if ((unsigned long long)rows > need) rows = (int)need;
    unsigned* partial = nullptr;
    e = cudaMallocAsync(&partial, (size_t)rows * bins_bytes, st);
    if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_designability: cudaMallocAsync(partials)");
    if (rc == HP_OK) {
      e = cudaFuncSetAttribute(hist_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bins_bytes);
      if (e == cudaSuccess) e = launch_hist(d_phen, count, S, partial, rows, err, d_hist, bins_bytes, st);
      if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_designability: launch");
      cudaFreeAsync(partial, st);
    }
  } else {
    e = cudaMemsetAsync(d_hist, 0, sizeof(uint64_t) * (size_t)(S + 1), st);
    if (e == cudaSuccess) {
      hist_global<<<sm_count() * 4, 512, 0, st>>>(d_phen, count, S, reinterpret_cast<unsigned long long*>(d_hist), err);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_designability: launch");
  }
  return finish_with_err(err, st, "hp_designability", rc);
}

extern "C" int hp_robustness(const int32_t* d_phen, int32_t N, int32_t S, uint64_t* d_neutral, uint64_t* d_to_del,
                             void* stream) {
  if (!d_phen || !d_neutral || !d_to_del) return hp::fail(HP_EINVAL, "hp_robustness: NULL pointer");
  if (N < 1 || N > 40) return hp::fail(HP_EINVAL, "hp_robustness: N must be in [1, 40]");
  if (S < 1) return hp::fail(HP_EINVAL, "hp_robustness: S must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* err = nullptr;
  cudaError_t e = cudaMallocAsync(&err, 16, st);
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_robustness: cudaMallocAsync");
  unsigned long long* negcount = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(err) + 8);
  cudaMemsetAsync(err, 0, 16, st);
  cudaMemsetAsync(d_neutral, 0, sizeof(uint64_t) * (size_t)(S + 1), st);
  cudaMemsetAsync(d_to_del, 0, sizeof(uint64_t) * (size_t)(S + 1), st);
  e = hp::launch_robustness(d_phen, N, S, reinterpret_cast<unsigned long long*>(d_neutral),
                            reinterpret_cast<unsigned long long*>(d_to_del), negcount, err, st);
  const int rc = e == cudaSuccess ? HP_OK : hp::cuda_fail(e, "hp_robustness: launch");
  return finish_with_err(err, st, "hp_robustness", rc);
}

namespace hp {

// The passes over the flips of an N-bit map: bits [0, k) first, then the high bits [k, N) in
// near-equal groups of at most kRobMaxPassBits, each with the kRobTileBits - h lowest bits
// contiguous (k = min(N, kRobTileBits)).
std::vector<RobPass> flip_passes(int N) {
  const int k = std::min((int)N, kRobTileBits);
  std::vector<RobPass> plan;
  {
    RobPass p{};
    p.c = k;
    p.h = 0;
    p.first = 1;
    for (int b = k; b < N; b++) p.rest[p.nrest++] = b;
    plan.push_back(p);
  }
  const int R = N - k;
  const int np = (R + kRobMaxPassBits - 1) / kRobMaxPassBits;
  for (int i = 0, lo = k; i < np; i++) {
    RobPass p{};
    p.h = R / np + (i < R % np ? 1 : 0);
    p.c = kRobTileBits - p.h;
    for (int t = 0; t < p.h; t++) p.pos[t] = lo + t;
    for (int b = p.c; b < N; b++)
      if (b < lo || b >= lo + p.h) p.rest[p.nrest++] = b;
    lo += p.h;
    plan.push_back(p);
  }
  return plan;
}

cudaError_t launch_robustness(const int32_t* d_phen, int N, int S, unsigned long long* neutral,
                              unsigned long long* to_del, unsigned long long* negcount, unsigned* err, cudaStream_t st) {
  const int k = std::min((int)N, kRobTileBits);
  const unsigned long long blocks = 1ull << (N - k);
  const size_t smem = 2 * (sizeof(int32_t) << kRobTileBits) + (sizeof(uint16_t) << kRobTileBits);
  cudaError_t e = cudaFuncSetAttribute(robustness_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const std::vector<RobPass> plan = flip_passes(N);
  // a few CTAs per SM walking the blocks (shared memory: two blocks each), counting into
  // replicated counters (stream-ordered scratch; without it, straight into neutral / to_del)
  const unsigned grid = (unsigned)std::min<unsigned long long>(blocks, (unsigned long long)sm_count() * 2);
  unsigned long long* rep = nullptr;
  const size_t rep_bytes = sizeof(unsigned long long) * 2 * kRobReplicas * (size_t)S;
  if (cudaMallocAsync(&rep, rep_bytes, st) != cudaSuccess || cudaMemsetAsync(rep, 0, rep_bytes, st) != cudaSuccess) {
    if (rep) cudaFreeAsync(rep, st);
    rep = nullptr;
    cudaGetLastError();  // clear the failed allocation's error
  }
  for (const RobPass& p : plan) {
    if (rep)
      robustness_pass<<<grid, kRobThreads, smem, st>>>(d_phen, S, p, blocks, kRobReplicas, rep, rep + (size_t)kRobReplicas * S,
                                                       negcount, err);
    else
      robustness_pass<<<grid, kRobThreads, smem, st>>>(d_phen, S, p, blocks, 1, neutral, to_del, negcount, err);
  }
  if (rep) {
    robustness_gather<<<(S + 255) / 256, 256, 0, st>>>(rep, kRobReplicas, S, neutral, to_del);
    cudaFreeAsync(rep, st);
  }
  robustness_finish<<<1, 1024, 0, st>>>(N, S, neutral, to_del, negcount);
  return cudaGetLastError();
}

}  // namespace hp

extern "C" int hp_neutral_components(const int32_t* d_phen, int32_t N, int32_t S, int32_t* d_label, uint64_t* d_ncomp,
                                     void* stream) {
  if (!d_phen || !d_label || !d_ncomp) return hp::fail(HP_EINVAL, "hp_neutral_components: NULL pointer");
  if (N < 1 || N > 31) return hp::fail(HP_EUNSUPPORTED, "hp_neutral_components: N must be in [1, 31]");
  if (S < 1) return hp::fail(HP_EINVAL, "hp_neutral_components: S must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* err = nullptr;
  cudaError_t e = cudaMallocAsync(&err, sizeof(unsigned), st);
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_neutral_components: cudaMallocAsync");
  cudaMemsetAsync(err, 0, sizeof(unsigned), st);
  cudaMemsetAsync(d_ncomp, 0, sizeof(uint64_t) * (size_t)S, st);
  const unsigned long long total = 1ull << N;
  const unsigned grid = (unsigned)std::min<unsigned long long>((total + 255) / 256, (unsigned long long)sm_count() * 16);
  cc_init<<<grid, 256, 0, st>>>(d_phen, total, S, d_label, err);
  cc_hook<<<grid, 256, 0, st>>>(d_phen, N, d_label, err);
  cc_finish<<<grid, 256, 0, st>>>(d_phen, total, d_label, reinterpret_cast<unsigned long long*>(d_ncomp));
  e = cudaGetLastError();
  int rc = e == cudaSuccess ? HP_OK : hp::cuda_fail(e, "hp_neutral_components: launch");
  return finish_with_err(err, st, "hp_neutral_components", rc);
}

// ---------------------------------------------------------------- designability without allocation
//
// Some callers cannot let a library allocate device memory: a process whose
// framework or service has already reserved the device's memory in its own
// pool (where cudaMalloc / cudaMallocAsync would fail or fragment that pool),
// or code with a fixed device-memory budget.  For them the partial histograms
// and the error word of the designability pass live in one file-scope device
// array instead of per-call allocations.  Host code may not pass the array's
// name to a kernel (that is a host-side stand-in, not a device address): its
// device address is looked up once per device with cudaGetSymbolAddress.

namespace {

constexpr size_t kNoAllocWords = 1u << 20;  // 4 MiB of scratch, held by every GPU that loads the library
constexpr size_t kNoAllocHeader = 64;       // word 0: error word; partial rows start 256 bytes in
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned g_noalloc_scratch[kNoAllocWords];

std::mutex g_noalloc_mu;
unsigned* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};
unsigned long long g_noalloc_ctx[kNoAllocMaxDevices] = {0};  // id of the context the address belongs to

// Unique id of the current CUDA context (0 if the driver cannot tell).  A device reset destroys
// the context and the module with its array; the next context gets a new id, so an address
// looked up in the old context is never reused.  The driver calls are reached through the
// runtime's entry-point query, so the library does not link libcuda itself.
unsigned long long current_context_id() {
  typedef CUresult (*get_current_fn)(CUcontext*);
  typedef CUresult (*get_id_fn)(CUcontext, unsigned long long*);
  static get_current_fn get_current = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    return cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess
               ? reinterpret_cast<get_current_fn>(f)
               : nullptr;
  }();
  static get_id_fn get_id = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    return cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess
               ? reinterpret_cast<get_id_fn>(f)
               : nullptr;
  }();
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current context: looked up (cudaGetSymbolAddress)
// on the first call in each context of each device, then cached under the context's id.
int noalloc_scratch(unsigned** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_designability_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices) return hp::fail(HP_EUNSUPPORTED, "hp_designability_noalloc: device index too large");
  // 0 (no context bound to this thread yet, or no answer from the driver) always looks the address up
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev] || ctx == 0 || g_noalloc_ctx[dev] != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return hp::cuda_fail(e, "hp_designability_noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = static_cast<unsigned*>(p);
    g_noalloc_ctx[dev] = ctx;
  }
  *out = g_noalloc_ptr[dev];
  return HP_OK;
}

}  // namespace

extern "C" int hp_designability_noalloc(const int32_t* d_phen, uint64_t count, int32_t S, uint64_t* d_hist,
                                        void* stream) {
  if (!d_phen || !d_hist) return hp::fail(HP_EINVAL, "hp_designability_noalloc: NULL pointer");
  if (S < 1) return hp::fail(HP_EINVAL, "hp_designability_noalloc: S must be >= 1");
  int dev = 0, max_smem = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_designability_noalloc: cudaGetDevice");
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t bins = (size_t)S + 1;
  const size_t bins_bytes = bins * sizeof(unsigned);
  if (bins_bytes > (size_t)max_smem || bins > kNoAllocWords - kNoAllocHeader)
    return hp::fail(HP_EINVAL, "hp_designability_noalloc: S + 1 = " + std::to_string(bins) +
                                   " bins exceed the limit of this entry point (" +
                                   std::to_string(std::min((size_t)max_smem / sizeof(unsigned), kNoAllocWords - kNoAllocHeader)) +
                                   " bins: one shared-memory histogram and the 4 MiB static scratch)");
  unsigned* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != HP_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* err = scratch;
  unsigned* partial = scratch + kNoAllocHeader;
  int rows = (int)std::min<size_t>((size_t)sm_count(), (kNoAllocWords - kNoAllocHeader) / bins);
  const unsigned long long need = (count + kHistThreads * 4ull - 1) / (kHistThreads * 4ull);
  if ((unsigned long long)rows > need) rows = (int)std::max<unsigned long long>(need, 1ull);
  // the error word starts at zero; every partial row is fully overwritten by its CTA
  e = cudaMemsetAsync(err, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_designability_noalloc: cudaMemsetAsync");
  if (count == 0) {
    e = cudaMemsetAsync(d_hist, 0, sizeof(uint64_t) * bins, st);
  } else {
    e = cudaFuncSetAttribute(hist_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bins_bytes);
    if (e == cudaSuccess) e = launch_hist(d_phen, count, S, partial, rows, err, d_hist, bins_bytes, st);
  }
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_designability_noalloc: launch");
  unsigned herr = 0;
  e = cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_designability_noalloc: execution");
  if (herr & kErrRange) return hp::fail(HP_EINVAL, "hp_designability_noalloc: map entry outside [-1, S)");
  return HP_OK;
}

// ---------------------------------------------------------------- one row of Eq. 2

namespace {

// out[p] += #{(g, i) : P(g) = q, P(g xor 2^i) = p} over a full 2^N map (index S for -1).  The
// row is sparse (a phenotype's neighbours are few), so it is accumulated with global atomics
// issued only by genotypes of phenotype q.
__global__ void neighbourhood_row(const int32_t* __restrict__ phen, int N, int S, int32_t q,
                                  unsigned long long* __restrict__ out, unsigned* __restrict__ err) {
  const unsigned long long total = 1ull << N;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    if (__ldcs(phen + g) != q) continue;
    for (int i = 0; i < N; i++) {
      const int32_t p = __ldg(phen + (g ^ (1ull << i)));
      if (p < -1 || p >= S) {
        atomicOr(err, kErrRange);
        continue;
      }
      atomicAdd(&out[p < 0 ? S : p], 1ull);
    }
  }
}

}  // namespace

extern "C" int hp_neighbourhood(const int32_t* d_phen, int32_t N, int32_t S, int32_t q, uint64_t* d_row, void* stream) {
  if (!d_phen || !d_row) return hp::fail(HP_EINVAL, "hp_neighbourhood: NULL pointer");
  if (N < 1 || N > 40) return hp::fail(HP_EINVAL, "hp_neighbourhood: N must be in [1, 40]");
  if (S < 1 || q < -1 || q >= S) return hp::fail(HP_EINVAL, "hp_neighbourhood: q must be in [-1, S)");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* err = nullptr;
  cudaError_t e = cudaMallocAsync(&err, sizeof(unsigned), st);
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_neighbourhood: cudaMallocAsync");
  cudaMemsetAsync(err, 0, sizeof(unsigned), st);
  cudaMemsetAsync(d_row, 0, sizeof(uint64_t) * (size_t)(S + 1), st);
  const unsigned long long total = 1ull << N;
  const unsigned grid = (unsigned)std::min<unsigned long long>((total + 255) / 256, (unsigned long long)sm_count() * 16);
  neighbourhood_row<<<grid, 256, 0, st>>>(d_phen, N, S, q, reinterpret_cast<unsigned long long*>(d_row), err);
  e = cudaGetLastError();
  int rc = e == cudaSuccess ? HP_OK : hp::cuda_fail(e, "hp_neighbourhood: launch");
  return finish_with_err(err, st, "hp_neighbourhood", rc);
}

// ---------------------------------------------------------------- cross-block flips

namespace {

// Genotypes of block A (ids base_a + x) flipped across one high bit land on base_b + x in block B:
// neutral[P_A(x)] += [P_B(x) = P_A(x)], to_del[P_A(x)] += [P_B(x) = -1]  (index S for -1).
__global__ void robustness_cross(const int32_t* __restrict__ a, const int32_t* __restrict__ b, unsigned long long count,
                                 int S, unsigned long long* __restrict__ neutral, unsigned long long* __restrict__ to_del,
                                 unsigned* __restrict__ err) {
  unsigned negneg = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < count; x += stride) {
    const int32_t pa = __ldcs(a + x), pb = __ldcs(b + x);
    if (pa < -1 || pa >= S || pb < -1 || pb >= S) {
      atomicOr(err, kErrRange);
      continue;
    }
    if (pa < 0) {
      negneg += pb < 0;
    } else if (pb == pa) {
      atomicAdd(&neutral[pa], 1ull);
    } else if (pb < 0) {
      atomicAdd(&to_del[pa], 1ull);
    }
  }
  for (int off = 16; off; off >>= 1) negneg += __shfl_xor_sync(0xFFFFFFFFu, negneg, off);
  if ((threadIdx.x & 31) == 0 && negneg) {
    atomicAdd(&neutral[S], (unsigned long long)negneg);
    atomicAdd(&to_del[S], (unsigned long long)negneg);
  }
}

}  // namespace

extern "C" int hp_robustness_cross(const int32_t* d_phen_a, const int32_t* d_phen_b, uint64_t count, int32_t S,
                                   uint64_t* d_neutral, uint64_t* d_to_del, void* stream) {
  if (!d_phen_a || !d_phen_b || !d_neutral || !d_to_del) return hp::fail(HP_EINVAL, "hp_robustness_cross: NULL pointer");
  if (S < 1) return hp::fail(HP_EINVAL, "hp_robustness_cross: S must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* err = nullptr;
  cudaError_t e = cudaMallocAsync(&err, sizeof(unsigned), st);
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_robustness_cross: cudaMallocAsync");
  cudaMemsetAsync(err, 0, sizeof(unsigned), st);
  int rc = HP_OK;
  if (count) {
    const unsigned grid = (unsigned)std::min<unsigned long long>((count + 255) / 256, (unsigned long long)sm_count() * 16);
    robustness_cross<<<grid, 256, 0, st>>>(d_phen_a, d_phen_b, count, S, reinterpret_cast<unsigned long long*>(d_neutral),
                                            reinterpret_cast<unsigned long long*>(d_to_del), err);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_robustness_cross: launch");
  }
  return finish_with_err(err, st, "hp_robustness_cross", rc);
}
