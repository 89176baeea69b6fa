// Neutral networks of a sequence space too large for one label array (the 6x6 space of 2^36
// genotypes): connected components of the graph on {g : P(g) != -1} with edges g -- g xor 2^i where
// the phenotypes are equal (Section 1; the paper does not compute them), counted per phenotype.
//
// The space is split by its top b bits into 2^b shards of 2^m ids (m = N - b), as in the shard
// streamer.  Inside a shard the flips of the m low bits give local components (the union-find of
// hp_neutral_components over the shard as a space of its own); a local component is named by its
// smallest global id, (k << m) + its smallest offset.  A flip of shard bit t joins offset x of shard
// j to offset x of shard j xor 2^t; when both ends fold to the same phenotype it joins their local
// components.  Per pair of neighbouring shards a kernel collects the DISTINCT pairs of local
// component names joined this way (a device hash set), and a host union-find over all local
// components merges them.  The number of components of phenotype p is the number of its merged
// classes.  Shard maps stay resident while a neighbour still needs them (window >= 2^(b-1) + 1, as
// for the streamer); local labels are recomputed from a resident map when a pair needs them (the
// union-find of one 2^28-id 6x6 shard takes about 35 ms, its map 0.65 s).
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "hp_internal.h"

extern "C" int hp_phenotype_map(const hp_structs* s, uint64_t seq_begin, uint64_t seq_count, int32_t gap_threshold,
                                int32_t* d_phen, int32_t* d_argmin_aux, void* stream);
extern "C" int hp_neutral_components(const int32_t* d_phen, int32_t N, int32_t S, int32_t* d_label, uint64_t* d_ncomp,
                                     void* stream);

namespace {

constexpr unsigned long long kEmptyPair = ~0ull;
constexpr unsigned kErrFull = 1u;

// local roots of a shard: offsets x with label[x] == x (the smallest member of a local component)
// and their phenotypes; *n counts them, entries beyond cap are only counted
__global__ void local_roots(const int32_t* __restrict__ phen, const int32_t* __restrict__ label, unsigned long long count,
                            unsigned* __restrict__ out_x, int32_t* __restrict__ out_p, unsigned long long cap,
                            unsigned long long* n) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < count; x += stride) {
    if (__ldcs(label + x) != (int32_t)x) continue;
    const unsigned long long at = atomicAdd(n, 1ull);
    if (at < cap) {
      out_x[at] = (unsigned)x;
      out_p[at] = phen[x];
    }
  }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z ^= z >> 33;
  z *= 0xff51afd7ed558ccdull;
  z ^= z >> 33;
  return z;
}

// distinct (label_a[x], label_b[x]) over the offsets x where both maps fold to the same phenotype
__global__ void cross_pairs(const int32_t* __restrict__ pa, const int32_t* __restrict__ la, const int32_t* __restrict__ pb,
                            const int32_t* __restrict__ lb, unsigned long long count, unsigned long long* table,
                            int log2cap, unsigned* err) {
  const unsigned long long mask = (1ull << log2cap) - 1ull;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < count; x += stride) {
    const int32_t p = __ldcs(pa + x);
    if (p < 0 || __ldcs(pb + x) != p) continue;
    const unsigned long long key = ((unsigned long long)(uint32_t)__ldcs(la + x) << 32) | (uint32_t)__ldcs(lb + x);
    unsigned long long s = mix64(key) & mask;
    bool done = false;
    for (unsigned long long probe = 0; probe <= mask && !done; probe++, s = (s + 1) & mask) {
      unsigned long long k = table[s];
      if (k == kEmptyPair) k = atomicCAS(table + s, kEmptyPair, key);
      done = k == kEmptyPair || k == key;
    }
    if (!done) atomicOr(err, kErrFull);
  }
}

__global__ void compact_pairs(const unsigned long long* __restrict__ table, unsigned long long cap,
                              unsigned long long* __restrict__ out, unsigned long long* n) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += stride) {
    const unsigned long long k = table[s];
    if (k != kEmptyPair) out[atomicAdd(n, 1ull)] = k;
  }
}

int grid_for(unsigned long long n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (int)std::min<unsigned long long>((n + 255) / 256, (unsigned long long)std::max(sms, 1) * 16);
}

struct Dsu {
  std::vector<int32_t> parent;
  int32_t find(int32_t x) {
    while (parent[x] != x) {
      parent[x] = parent[parent[x]];
      x = parent[x];
    }
    return x;
  }
  void unite(int32_t a, int32_t b) {
    a = find(a);
    b = find(b);
    if (a != b) parent[std::max(a, b)] = std::min(a, b);
  }
};

}  // namespace

extern "C" int hp_stream_components(const hp_structs* s, int32_t shard_bits, int32_t window, uint64_t* h_ncomp,
                                    int32_t* h_maps_computed, void* stream) {
  if (!s || !h_ncomp) return hp::fail(HP_EINVAL, "hp_stream_components: NULL argument");
  const int b = shard_bits, N = s->N, m = N - b;
  if (b < 0 || b > 16 || m < 1 || m > 31)
    return hp::fail(HP_EINVAL, "hp_stream_components: shard_bits must be in [max(0, N-31), min(16, N-1)]");
  const int nsh = 1 << b;
  const int need_window = b == 0 ? 1 : (1 << (b - 1)) + 1;
  if (window < need_window)
    return hp::fail(HP_EINVAL,
                    "hp_stream_components: window must be at least 2^(shard_bits-1) + 1 = " + std::to_string(need_window));
  if (window > nsh) window = nsh;
  const int S = s->S;
  const unsigned long long shard_ids = 1ull << m;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = HP_OK;
  cudaError_t e = cudaSuccess;
  // device: window maps, two label buffers, local-component counts, a root list and a pair set
  std::vector<int32_t*> slots(window, nullptr);
  std::vector<int> slot_of(nsh, -1), owner(window, -1);
  std::vector<int> pending(nsh, 0);  // neighbours j > k whose pairs with k are still to do
  for (int k = 0; k < nsh; k++)
    for (int t = 0; t < b; t++) pending[k] += (k ^ (1 << t)) > k;
  int32_t* lab[2] = {nullptr, nullptr};
  uint64_t* dncomp = nullptr;
  unsigned long long* dn = nullptr;  // [0] roots, [1] pairs
  unsigned* derr = nullptr;
  unsigned* rx = nullptr;
  int32_t* rp = nullptr;
  unsigned long long* table = nullptr;
  unsigned long long* pairs = nullptr;
  unsigned long long root_cap = 1ull << 20, log2pairs = 22;
  e = cudaMalloc(&lab[0], shard_ids * 4);
  if (e == cudaSuccess) e = cudaMalloc(&lab[1], shard_ids * 4);
  if (e == cudaSuccess) e = cudaMalloc(&dncomp, (size_t)S * 8);
  if (e == cudaSuccess) e = cudaMalloc(&dn, 16);
  if (e == cudaSuccess) e = cudaMalloc(&derr, 4);
  if (e == cudaSuccess) e = cudaMalloc(&rx, root_cap * 4);
  if (e == cudaSuccess) e = cudaMalloc(&rp, root_cap * 4);
  if (e == cudaSuccess) e = cudaMalloc(&table, (1ull << log2pairs) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&pairs, (1ull << log2pairs) * 8);
  if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_stream_components: device buffers");
  // host: local components of every shard (sorted by offset; node = shard base + rank in the
  // shard) and a union-find over them, joined as the pairs arrive
  std::vector<std::vector<unsigned>> roots(nsh);
  std::vector<std::vector<int32_t>> root_p(nsh);
  std::vector<unsigned long long> node_base(nsh + 1, 0);
  Dsu d;
  auto node_of = [&](int k, unsigned x) -> int64_t {
    const std::vector<unsigned>& r = roots[k];
    const auto it = std::lower_bound(r.begin(), r.end(), x);
    if (it == r.end() || *it != x) return -1;
    return (int64_t)node_base[k] + (it - r.begin());
  };
  int computed = 0;
  // labels of the shard in `slot` into lab[which]
  auto labels = [&](int slot, int which) {
    return hp_neutral_components(slots[slot], m, S, lab[which], dncomp, st);
  };
  for (int k = 0; k < nsh && rc == HP_OK; k++) {
    int slot = -1;
    for (int q = 0; q < window && slot < 0; q++)
      if (owner[q] < 0 || pending[owner[q]] == 0) slot = q;
    if (slot < 0) {
      rc = hp::fail(HP_EINVAL, "hp_stream_components: window too small");
      break;
    }
    if (owner[slot] >= 0) slot_of[owner[slot]] = -1;
    if (!slots[slot]) {
      e = cudaMalloc(&slots[slot], shard_ids * 4);
      if (e != cudaSuccess) {
        rc = hp::cuda_fail(e, "hp_stream_components: shard map buffer");
        break;
      }
    }
    owner[slot] = k;
    slot_of[k] = slot;
    rc = hp_phenotype_map(s, (unsigned long long)k << m, shard_ids, 1, slots[slot], nullptr, st);
    if (rc != HP_OK) break;
    computed++;
    // local components of shard k: labels into lab[0], roots to the host
    rc = labels(slot, 0);
    if (rc != HP_OK) break;
    for (int attempt = 0; attempt < 2 && rc == HP_OK; attempt++) {
      unsigned long long nroots = 0;
      cudaMemsetAsync(dn, 0, 16, st);
      local_roots<<<grid_for(shard_ids), 256, 0, st>>>(slots[slot], lab[0], shard_ids, rx, rp, root_cap, dn);
      e = cudaMemcpyAsync(&nroots, dn, 8, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        rc = hp::cuda_fail(e, "hp_stream_components: local roots");
        break;
      }
      if (nroots > root_cap) {  // grow the list once to the exact count and run again
        cudaFree(rx);
        cudaFree(rp);
        root_cap = nroots;
        e = cudaMalloc(&rx, root_cap * 4);
        if (e == cudaSuccess) e = cudaMalloc(&rp, root_cap * 4);
        if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_stream_components: root list");
        continue;
      }
      std::vector<unsigned> x(nroots);
      std::vector<int32_t> p(nroots);
      e = cudaMemcpy(x.data(), rx, nroots * 4, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(p.data(), rp, nroots * 4, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        rc = hp::cuda_fail(e, "hp_stream_components: root list read back");
        break;
      }
      std::vector<size_t> order(nroots);
      std::iota(order.begin(), order.end(), 0);
      std::sort(order.begin(), order.end(), [&](size_t a, size_t c) { return x[a] < x[c]; });
      roots[k].resize(nroots);
      root_p[k].resize(nroots);
      for (size_t i = 0; i < nroots; i++) {
        roots[k][i] = x[order[i]];
        root_p[k][i] = p[order[i]];
      }
      node_base[k + 1] = node_base[k] + nroots;
      if (node_base[k + 1] >= 0x7FFFFFFFull) {
        rc = hp::fail(HP_EUNSUPPORTED, "hp_stream_components: more than 2^31 local components");
        break;
      }
      const size_t old = d.parent.size();
      d.parent.resize(node_base[k + 1]);
      std::iota(d.parent.begin() + old, d.parent.end(), (int32_t)old);
      break;
    }
    if (rc != HP_OK) break;
    // joins with every lower neighbour j (resident: its pending count was not yet zero)
    for (int t = 0; t < b && rc == HP_OK; t++) {
      const int j = k ^ (1 << t);
      if (j > k) continue;
      if (slot_of[j] < 0) {
        rc = hp::fail(HP_EINVAL, "hp_stream_components: a neighbour map left the window");
        break;
      }
      rc = labels(slot_of[j], 1);
      if (rc != HP_OK) break;
      for (int attempt = 0; attempt < 8 && rc == HP_OK; attempt++) {
        const unsigned long long cap = 1ull << log2pairs;
        unsigned herr = 0;
        unsigned long long npairs = 0;
        cudaMemsetAsync(table, 0xFF, cap * 8, st);
        cudaMemsetAsync(dn, 0, 16, st);
        cudaMemsetAsync(derr, 0, 4, st);
        cross_pairs<<<grid_for(shard_ids), 256, 0, st>>>(slots[slot_of[j]], lab[1], slots[slot], lab[0], shard_ids, table,
                                                         (int)log2pairs, derr);
        e = cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
          rc = hp::cuda_fail(e, "hp_stream_components: cross pairs");
          break;
        }
        if (herr & kErrFull) {  // more distinct joins than slots: a table twice the size, again
          cudaFree(table);
          cudaFree(pairs);
          table = pairs = nullptr;
          log2pairs++;
          e = cudaMalloc(&table, (1ull << log2pairs) * 8);
          if (e == cudaSuccess) e = cudaMalloc(&pairs, (1ull << log2pairs) * 8);
          if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_stream_components: pair table");
          continue;
        }
        compact_pairs<<<grid_for(cap), 256, 0, st>>>(table, cap, pairs, dn + 1);
        e = cudaMemcpyAsync(&npairs, dn + 1, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        std::vector<unsigned long long> hp_pairs(npairs);
        if (e == cudaSuccess) e = cudaMemcpy(hp_pairs.data(), pairs, npairs * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
          rc = hp::cuda_fail(e, "hp_stream_components: pair read back");
          break;
        }
        for (unsigned long long key : hp_pairs) {
          const int64_t a = node_of(j, (unsigned)(key >> 32)), c = node_of(k, (unsigned)(key & 0xFFFFFFFFu));
          if (a < 0 || c < 0) {
            rc = hp::fail(HP_EINVAL, "hp_stream_components: a join names an unknown local component");
            break;
          }
          d.unite((int32_t)a, (int32_t)c);
        }
        break;
      }
      pending[j]--;
    }
  }
  for (int32_t* p : slots) cudaFree(p);
  cudaFree(lab[0]);
  cudaFree(lab[1]);
  cudaFree(dncomp);
  cudaFree(dn);
  cudaFree(derr);
  cudaFree(rx);
  cudaFree(rp);
  cudaFree(table);
  cudaFree(pairs);
  if (rc != HP_OK) return rc;
  std::fill(h_ncomp, h_ncomp + S, 0ull);
  for (int k = 0; k < nsh; k++)
    for (size_t i = 0; i < roots[k].size(); i++) {
      const int32_t node = (int32_t)(node_base[k] + i);
      const int32_t p = root_p[k][i];
      if (p < 0 || p >= S) return hp::fail(HP_EINVAL, "hp_stream_components: a local root with no phenotype");
      if (d.find(node) == node) h_ncomp[p]++;
    }
  if (h_maps_computed) *h_maps_computed = computed;
  return HP_OK;
}
