// Shard streamer: the map of a large sequence space (the paper's 6x6 run of
// 2^36 genotypes, Sections 3.1 and 4) computed shard by shard, with exact
// integer designability and Eq. 2 numerators, a bounded window of resident
// shard maps, and per-shard records on disk so that an interrupted run resumes.
//
// The space [0, 2^N) is split by its top b bits into 2^b shards of 2^m ids
// (m = N - b).  Flips of the m low bits stay inside a shard; a flip of bit
// m + t joins shard k to shard k xor 2^t at the same offset.  Records:
//   in_<k>           designability and in-shard numerators of shard k
//   cross_<j>_<k>    numerators of j's genotypes flipped into k and of k's into j
// The totals are the exact sums of all records and equal the single-pass
// reductions of the full map.  A shard map is computed only if one of its
// records is missing and stays resident until all its cross records exist;
// visiting shards in increasing order needs 2^(b-1) + 1 resident maps.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <sys/stat.h>
#include <vector>

#include "hp_internal.h"

extern "C" int hp_designability(const int32_t* d_phen, uint64_t count, int32_t S, uint64_t* d_hist, void* stream);
extern "C" int hp_robustness(const int32_t* d_phen, int32_t N, int32_t S, uint64_t* d_neutral, uint64_t* d_to_del,
                             void* stream);
extern "C" int hp_robustness_cross(const int32_t* d_phen_a, const int32_t* d_phen_b, uint64_t count, int32_t S,
                                   uint64_t* d_neutral, uint64_t* d_to_del, void* stream);
extern "C" int hp_phenotype_map(const hp_structs* s, uint64_t seq_begin, uint64_t seq_count, int32_t gap_threshold,
                                int32_t* d_phen, int32_t* d_argmin_aux, void* stream);

namespace {

uint64_t table_hash(const hp_structs* s) {
  uint64_t h = 1469598103934665603ull;  // FNV-1a, 64-bit
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; i++) {
      h ^= c[i];
      h *= 1099511628211ull;
    }
  };
  mix(s->L, sizeof(s->L));
  mix(s->conf.data(), s->conf.size());
  mix(s->conf_class.data(), s->conf_class.size() * sizeof(int32_t));
  return h;
}

struct Record {
  std::vector<uint64_t> v;  // concatenated counter rows
  bool have = false;
};

// FNV-1a (64-bit) of a record's counters, stored in its header: a record whose payload does not
// match (a flipped bit, a torn or foreign file) is not reused, so its shard is computed again.
uint64_t payload_sum(const std::vector<uint64_t>& v) {
  uint64_t h = 1469598103934665603ull;
  const unsigned char* c = reinterpret_cast<const unsigned char*>(v.data());
  for (size_t i = 0; i < v.size() * sizeof(uint64_t); i++) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

// header: table hash, payload words, payload checksum
bool read_record(const std::string& path, uint64_t hash, size_t words, Record& r) {
  FILE* f = fopen(path.c_str(), "rb");
  if (!f) return false;
  uint64_t hdr[3] = {0, 0, 0};
  r.v.assign(words, 0);
  bool ok = fread(hdr, 8, 3, f) == 3 && hdr[0] == hash && hdr[1] == words && fread(r.v.data(), 8, words, f) == words;
  unsigned char extra;
  ok = ok && fread(&extra, 1, 1, f) == 0 && payload_sum(r.v) == hdr[2];
  fclose(f);
  r.have = ok;
  if (!ok) r.v.clear();
  return ok;
}

bool write_record(const std::string& path, uint64_t hash, const std::vector<uint64_t>& v) {
  const std::string tmp = path + ".tmp";
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return false;
  const uint64_t hdr[3] = {hash, (uint64_t)v.size(), payload_sum(v)};
  bool ok = fwrite(hdr, 8, 3, f) == 3 && fwrite(v.data(), 8, v.size(), f) == v.size();
  ok = (fclose(f) == 0) && ok;
  return ok && rename(tmp.c_str(), path.c_str()) == 0;
}

}  // namespace

extern "C" int hp_stream_shards(const hp_structs* s, int32_t shard_bits, int32_t window, const char* out_dir,
                                uint64_t* h_hist, uint64_t* h_neutral, uint64_t* h_to_del, int32_t* h_maps_computed,
                                void* stream) {
  if (!s || !h_hist || !h_neutral || !h_to_del) return hp::fail(HP_EINVAL, "hp_stream_shards: NULL argument");
  const int b = shard_bits, N = s->N, m = N - b;
  if (b < 0 || b > 16 || m < 1) return hp::fail(HP_EINVAL, "hp_stream_shards: shard_bits must be in [0, min(16, N-1)]");
  const int nsh = 1 << b;
  const int need_window = b == 0 ? 1 : (1 << (b - 1)) + 1;
  if (window < need_window)
    return hp::fail(HP_EINVAL, "hp_stream_shards: window must be at least 2^(shard_bits-1) + 1 = " + std::to_string(need_window));
  if (window > nsh) window = nsh;
  const int S = s->S;
  const size_t W = (size_t)S + 1;
  const uint64_t hash = table_hash(s);
  const uint64_t shard_ids = 1ull << m;
  std::string dir = out_dir ? out_dir : "";
  if (!dir.empty()) {
    mkdir(dir.c_str(), 0755);
    FILE* f = fopen((dir + "/manifest.txt").c_str(), "w");
    if (!f) return hp::fail(HP_EINVAL, "hp_stream_shards: cannot write the manifest in " + dir);
    fprintf(f, "box %d %d %d\nN %d\nS %d\nS_dir %d\nshard_bits %d\nshard_ids %llu\ntable_hash %016llx\n", s->L[0], s->L[1],
            s->L[2], N, S, s->S_dir, b, (unsigned long long)shard_ids, (unsigned long long)hash);
    fclose(f);
  }
  auto in_path = [&](int k) { return dir + "/in_" + std::to_string(k) + ".bin"; };
  auto cross_path = [&](int j, int k) { return dir + "/cross_" + std::to_string(j) + "_" + std::to_string(k) + ".bin"; };
  // records already on disk
  std::vector<Record> rin(nsh);
  std::vector<std::vector<Record>> rcross(nsh, std::vector<Record>(b));  // rcross[k][t]: k with k ^ 2^t, k < partner
  for (int k = 0; k < nsh; k++) {
    if (!dir.empty()) read_record(in_path(k), hash, 3 * W, rin[k]);
    for (int t = 0; t < b; t++) {
      const int j = k ^ (1 << t);
      if (k < j && !dir.empty()) read_record(cross_path(k, j), hash, 4 * W, rcross[k][t]);
    }
  }
  auto cross_rec = [&](int k, int t) -> Record& {
    const int j = k ^ (1 << t);
    return k < j ? rcross[k][t] : rcross[j][t];
  };
  auto needed = [&](int k) {
    if (!rin[k].have) return true;
    for (int t = 0; t < b; t++)
      if (!cross_rec(k, t).have) return true;
    return false;
  };
  cudaStream_t st = (cudaStream_t)stream;
  // device buffers: `window` shard maps and counter rows
  std::vector<int32_t*> slots(window, nullptr);
  std::vector<int> slot_of(nsh, -1), owner(window, -1);
  uint64_t* dcnt = nullptr;  // 3 rows of W counters
  int rc = HP_OK;
  cudaError_t e = cudaMalloc(&dcnt, 3 * W * sizeof(uint64_t));
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_stream_shards: counters");
  int computed = 0;
  std::vector<uint64_t> host(4 * W);
  for (int k = 0; k < nsh && rc == HP_OK; k++) {
    if (!needed(k)) continue;
    // a free slot: evict maps whose records are all present
    int slot = -1;
    for (int q = 0; q < window && slot < 0; q++)
      if (owner[q] < 0 || !needed(owner[q])) slot = q;
    if (slot < 0) {
      rc = hp::fail(HP_EINVAL, "hp_stream_shards: window too small for the records still missing");
      break;
    }
    if (owner[slot] >= 0) slot_of[owner[slot]] = -1;
    if (!slots[slot]) {
      e = cudaMalloc(&slots[slot], shard_ids * sizeof(int32_t));
      if (e != cudaSuccess) {
        rc = hp::cuda_fail(e, "hp_stream_shards: shard map buffer");
        break;
      }
    }
    owner[slot] = k;
    slot_of[k] = slot;
    rc = hp_phenotype_map(s, (uint64_t)k << m, shard_ids, 1, slots[slot], nullptr, st);
    if (rc != HP_OK) break;
    computed++;
    if (!rin[k].have) {
      rc = hp_designability(slots[slot], shard_ids, S, dcnt, st);
      if (rc == HP_OK) rc = hp_robustness(slots[slot], m, S, dcnt + W, dcnt + 2 * W, st);
      if (rc != HP_OK) break;
      e = cudaMemcpyAsync(host.data(), dcnt, 3 * W * sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        rc = hp::cuda_fail(e, "hp_stream_shards: read back");
        break;
      }
      rin[k].v.assign(host.begin(), host.begin() + 3 * W);
      rin[k].have = true;
      if (!dir.empty() && !write_record(in_path(k), hash, rin[k].v)) rc = hp::fail(HP_EINVAL, "hp_stream_shards: record write failed");
    }
    // cross terms with lower neighbours (their maps are resident: they were needed for this record)
    for (int t = 0; t < b && rc == HP_OK; t++) {
      const int j = k ^ (1 << t);
      if (j > k || cross_rec(k, t).have) continue;
      if (slot_of[j] < 0) {
        rc = hp::fail(HP_EINVAL, "hp_stream_shards: a neighbour map left the window");
        break;
      }
      const int32_t* mj = slots[slot_of[j]];
      const int32_t* mk = slots[slot];
      cudaMemsetAsync(dcnt, 0, 2 * W * sizeof(uint64_t), st);
      rc = hp_robustness_cross(mj, mk, shard_ids, S, dcnt, dcnt + W, st);  // j's genotypes into k
      if (rc != HP_OK) break;
      e = cudaMemcpyAsync(host.data(), dcnt, 2 * W * sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      cudaMemsetAsync(dcnt, 0, 2 * W * sizeof(uint64_t), st);
      if (e == cudaSuccess) rc = hp_robustness_cross(mk, mj, shard_ids, S, dcnt, dcnt + W, st);  // k's into j
      if (e == cudaSuccess && rc == HP_OK) {
        e = cudaMemcpyAsync(host.data() + 2 * W, dcnt, 2 * W * sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      }
      if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_stream_shards: cross read back");
      if (rc != HP_OK) break;
      Record& r = cross_rec(k, t);
      r.v = host;
      r.have = true;
      if (!dir.empty() && !write_record(cross_path(j, k), hash, r.v)) rc = hp::fail(HP_EINVAL, "hp_stream_shards: record write failed");
    }
  }
  for (int32_t* p : slots) cudaFree(p);
  cudaFree(dcnt);
  if (rc != HP_OK) return rc;
  // exact totals: every record once
  std::memset(h_hist, 0, W * 8);
  std::memset(h_neutral, 0, W * 8);
  std::memset(h_to_del, 0, W * 8);
  for (int k = 0; k < nsh; k++) {
    for (size_t p = 0; p < W; p++) {
      h_hist[p] += rin[k].v[p];
      h_neutral[p] += rin[k].v[W + p];
      h_to_del[p] += rin[k].v[2 * W + p];
    }
    for (int t = 0; t < b; t++) {
      const int j = k ^ (1 << t);
      if (j < k) continue;
      const std::vector<uint64_t>& v = rcross[k][t].v;
      for (size_t p = 0; p < W; p++) {
        h_neutral[p] += v[p] + v[2 * W + p];
        h_to_del[p] += v[W + p] + v[3 * W + p];
      }
    }
  }
  if (h_maps_computed) *h_maps_computed = computed;
  return HP_OK;
}
