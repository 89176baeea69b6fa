// Fold library of a box: every compact self-avoiding walk (Hamiltonian path),
// reduced by the box's symmetry group G and by chain reversal (Section 2.1 of
// arXiv 2008.05612; the paper loads this library from a file and does not say
// how it was built).
//
// Construction used here:
//   * G is generated as the closure of two kinds of site permutations: the
//     reflection of each axis and the exchange of each pair of equal-length
//     axes.
//   * The walk search is a depth-first search that only ever extends a prefix
//     which is lexicographically minimal over its G-orbit: it tracks the set of
//     group elements that fix the prefix and refuses any next site that one of
//     them maps to a smaller site.  Every surviving complete walk is therefore
//     the canonical (smallest) member of its orbit, i.e. one directed
//     conformation.  A dead-end rule (a free site with no free neighbour other
//     than the head) prunes hopeless prefixes.
//   * Each conformation's reversal is canonicalised by brute force over G; the
//     class representative is the smaller of the two, classes are ranked by
//     representative and conformations ordered by (class, own tuple).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <set>

#include "hp_internal.h"

namespace {

struct Lattice {
  int L[3];
  int N;
  int nnb[hp::kMaxN];
  int nb[hp::kMaxN][6];
  void coords(int s, int c[3]) const {
    c[0] = s % L[0];
    c[1] = (s / L[0]) % L[1];
    c[2] = s / (L[0] * L[1]);
  }
  int site(const int c[3]) const { return c[0] + L[0] * (c[1] + L[1] * c[2]); }
};

using Perm = std::vector<uint8_t>;

std::vector<Perm> box_group(const Lattice& lat, int ndim) {
  std::vector<Perm> gens;
  for (int a = 0; a < ndim; a++) {  // reflections
    Perm p(lat.N);
    for (int s = 0; s < lat.N; s++) {
      int c[3];
      lat.coords(s, c);
      c[a] = lat.L[a] - 1 - c[a];
      p[s] = (uint8_t)lat.site(c);
    }
    gens.push_back(p);
  }
  for (int a = 0; a < ndim; a++)  // exchanges of equal-length axes
    for (int b = a + 1; b < ndim; b++) {
      if (lat.L[a] != lat.L[b]) continue;
      Perm p(lat.N);
      for (int s = 0; s < lat.N; s++) {
        int c[3];
        lat.coords(s, c);
        std::swap(c[a], c[b]);
        p[s] = (uint8_t)lat.site(c);
      }
      gens.push_back(p);
    }
  Perm id(lat.N);
  std::iota(id.begin(), id.end(), 0);
  std::set<Perm> seen{id};
  std::vector<Perm> order{id};
  for (size_t k = 0; k < order.size(); k++)
    for (const Perm& g : gens) {
      Perm h(lat.N);
      for (int s = 0; s < lat.N; s++) h[s] = g[order[k][s]];
      if (seen.insert(h).second) order.push_back(h);
    }
  return order;  // order[0] is the identity
}

struct Search {
  const Lattice* lat;
  const std::vector<Perm>* G;
  int N;
  uint8_t path[hp::kMaxN];
  bool used[hp::kMaxN];
  int freedeg[hp::kMaxN];  // unused neighbours of each site
  std::vector<uint8_t> out;
  int64_t found = 0;

  // Does visiting `t` next leave a free site that can no longer be reached?
  bool dead_end(int t, int remaining_after) const {
    if (remaining_after == 0) return false;
    int stuck = 0;
    for (int k = 0; k < lat->nnb[t]; k++) {
      int u = lat->nb[t][k];
      if (used[u]) continue;
      // after t is used, u keeps freedeg[u]-1 free neighbours (t removed)
      if (freedeg[u] - 1 == 0) stuck++;
    }
    // a free neighbour of the new head with no other free neighbour must be
    // visited next and must be the last site; two such neighbours cannot both be
    return stuck > 1 || (stuck == 1 && remaining_after > 1);
  }

  void visit(int t) {
    used[t] = true;
    for (int k = 0; k < lat->nnb[t]; k++) freedeg[lat->nb[t][k]]--;
  }
  void leave(int t) {
    used[t] = false;
    for (int k = 0; k < lat->nnb[t]; k++) freedeg[lat->nb[t][k]]++;
  }

  void dfs(int depth, uint64_t active) {
    if (depth == N) {
      out.insert(out.end(), path, path + N);
      found++;
      return;
    }
    int head = path[depth - 1];
    for (int k = 0; k < lat->nnb[head]; k++) {
      int t = lat->nb[head][k];
      if (used[t]) continue;
      uint64_t next = 0;
      bool smaller = false;
      for (uint64_t a = active; a; a &= a - 1) {
        int g = __builtin_ctzll(a);
        int gt = (*G)[g][t];
        if (gt < t) { smaller = true; break; }
        if (gt == t) next |= 1ull << g;
      }
      if (smaller) continue;
      if (dead_end(t, N - depth - 1)) continue;
      path[depth] = (uint8_t)t;
      visit(t);
      dfs(depth + 1, next);
      leave(t);
    }
  }
};

bool tuple_less(const uint8_t* a, const uint8_t* b, int n) {
  return std::lexicographical_compare(a, a + n, b, b + n);
}

}  // namespace

extern "C" int hp_enumerate_structures(int ndim, const int32_t dims[3], hp_structs** out) {
  if (!out) return hp::fail(HP_EINVAL, "hp_enumerate_structures: out is NULL");
  *out = nullptr;
  if (!dims) return hp::fail(HP_EINVAL, "hp_enumerate_structures: dims is NULL");
  if (ndim != 2 && ndim != 3) return hp::fail(HP_EINVAL, "hp_enumerate_structures: ndim must be 2 or 3");
  Lattice lat;
  int64_t n = 1;
  for (int k = 0; k < 3; k++) {
    lat.L[k] = k < ndim ? dims[k] : 1;
    if (lat.L[k] < 1) return hp::fail(HP_EINVAL, "hp_enumerate_structures: side lengths must be >= 1");
    n *= lat.L[k];
    if (n > 1 << 20) break;
  }
  if (n < 2) return hp::fail(HP_EINVAL, "hp_enumerate_structures: the box needs at least 2 sites");
  if (n > hp::kMaxN) return hp::fail(HP_EUNSUPPORTED, "hp_enumerate_structures: more than 40 sites");
  lat.N = (int)n;
  for (int s = 0; s < lat.N; s++) {
    lat.nnb[s] = 0;
    int c[3];
    lat.coords(s, c);
    for (int a = 0; a < 3; a++)
      for (int d = -1; d <= 1; d += 2) {
        int e[3] = {c[0], c[1], c[2]};
        e[a] += d;
        if (e[a] < 0 || e[a] >= lat.L[a]) continue;
        lat.nb[s][lat.nnb[s]++] = lat.site(e);
      }
  }
  std::vector<Perm> G = box_group(lat, ndim);
  if ((int)G.size() > hp::kMaxSym) return hp::fail(HP_EINVAL, "hp_enumerate_structures: symmetry group too large");

  hp_structs* st = new (std::nothrow) hp_structs();
  if (!st) return hp::fail(HP_ENOMEM, "hp_enumerate_structures: out of host memory");
  try {
    st->ndim = ndim;
    for (int k = 0; k < 3; k++) st->L[k] = lat.L[k];
    st->N = lat.N;
    st->NE = (lat.N + 1) / 2;
    st->NO = lat.N / 2;
    st->nsym = (int)G.size();
    int N = lat.N;

    Search sr;
    sr.lat = &lat;
    sr.G = &G;
    sr.N = N;
    for (int s = 0; s < N; s++) {
      sr.used[s] = false;
      sr.freedeg[s] = lat.nnb[s];
    }
    uint64_t all = G.size() == 64 ? ~0ull : ((1ull << G.size()) - 1);
    for (int s0 = 0; s0 < N; s0++) {
      uint64_t next = 0;
      bool smaller = false;
      for (size_t g = 0; g < G.size(); g++) {
        if (G[g][s0] < s0) { smaller = true; break; }
        if (G[g][s0] == s0) next |= 1ull << g;
      }
      if (smaller) continue;
      (void)all;
      sr.path[0] = (uint8_t)s0;
      sr.visit(s0);
      if (N == 1) {
        sr.out.push_back((uint8_t)s0);
        sr.found++;
      } else {
        sr.dfs(1, next);
      }
      sr.leave(s0);
    }
    int64_t Sdir = sr.found;
    if (Sdir == 0) {
      delete st;
      return hp::fail(HP_EINVAL, "hp_enumerate_structures: the box has no Hamiltonian path");
    }
    if (Sdir > INT32_MAX / 2) {
      delete st;
      return hp::fail(HP_EUNSUPPORTED, "hp_enumerate_structures: too many conformations");
    }

    // representative of each conformation's class: min(own, canonical reversal)
    std::vector<uint8_t> rep((size_t)Sdir * N);
    for (int64_t i = 0; i < Sdir; i++) {
      const uint8_t* p = &sr.out[(size_t)i * N];
      uint8_t best[hp::kMaxN], cand[hp::kMaxN];
      for (int k = 0; k < N; k++) best[k] = p[N - 1 - k];
      for (const Perm& g : G) {
        for (int k = 0; k < N; k++) cand[k] = g[p[N - 1 - k]];
        if (tuple_less(cand, best, N)) std::memcpy(best, cand, N);
      }
      const uint8_t* r = tuple_less(best, p, N) ? best : p;
      std::memcpy(&rep[(size_t)i * N], r, N);
    }
    std::vector<int64_t> idx((size_t)Sdir);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
      const uint8_t* ra = &rep[(size_t)a * N];
      const uint8_t* rb = &rep[(size_t)b * N];
      int c = std::memcmp(ra, rb, N);
      if (c != 0) return c < 0;
      return std::memcmp(&sr.out[(size_t)a * N], &sr.out[(size_t)b * N], N) < 0;
    });
    st->S_dir = (int32_t)Sdir;
    st->conf.resize((size_t)Sdir * N);
    st->conf_class.resize((size_t)Sdir);
    int32_t cls = -1;
    for (int64_t k = 0; k < Sdir; k++) {
      int64_t i = idx[(size_t)k];
      if (k == 0 || std::memcmp(&rep[(size_t)i * N], &rep[(size_t)idx[(size_t)k - 1] * N], N) != 0) cls++;
      st->conf_class[(size_t)k] = cls;
      std::memcpy(&st->conf[(size_t)k * N], &sr.out[(size_t)i * N], N);
    }
    st->S = cls + 1;

    // contacts and kernel records
    int box_edges = 0;
    for (int s = 0; s < N; s++) box_edges += lat.nnb[s];
    box_edges /= 2;
    st->C = box_edges - (N - 1);
    int C = st->C;
    st->contacts.assign((size_t)Sdir * (C > 0 ? C : 1) * 2, 0);
    st->rec_words = st->NE + 6;
    if (st->rec_words % 2 == 0) st->rec_words++;
    st->rec.assign((size_t)Sdir * st->rec_words, 0u);
    for (int64_t k = 0; k < Sdir; k++) {
      const uint8_t* p = &st->conf[(size_t)k * N];
      int pos[hp::kMaxN];
      for (int r = 0; r < N; r++) pos[p[r]] = r;
      int cnt = 0;
      int codd[hp::kMaxHalf] = {0};
      uint32_t* rec = &st->rec[(size_t)k * st->rec_words];
      for (int i = 0; i < N; i++) {
        int si = p[i];
        for (int q = 0; q < lat.nnb[si]; q++) {
          int j = pos[lat.nb[si][q]];
          if (j <= i + 1) continue;  // each pair once; skip chain bonds
          if (cnt >= C || ((i ^ j) & 1) == 0) {
            delete st;
            return hp::fail(HP_EINVAL, "hp_enumerate_structures: contact structure violates lattice bipartiteness");
          }
          st->contacts[((size_t)k * C + cnt) * 2] = (uint8_t)i;
          st->contacts[((size_t)k * C + cnt) * 2 + 1] = (uint8_t)j;
          cnt++;
          int ev = (i & 1) ? j : i, od = (i & 1) ? i : j;
          rec[ev / 2] |= 1u << (od / 2);
          codd[od / 2]++;
        }
      }
      if (cnt != C) {
        delete st;
        return hp::fail(HP_EINVAL, "hp_enumerate_structures: a walk does not have E - (N - 1) contacts");
      }
      // export order: contacts sorted by (i, j)
      uint16_t* pairs = reinterpret_cast<uint16_t*>(&st->contacts[(size_t)k * C * 2]);
      std::sort(pairs, pairs + C, [](uint16_t a, uint16_t b) {
        return ((a & 0xFF) << 8 | a >> 8) < ((b & 0xFF) << 8 | b >> 8);
      });
      for (int j = 0; j < st->NO; j++)
        for (int b = 0; b < 3; b++)
          if ((codd[j] >> b) & 1) rec[st->NE + b] |= 1u << j;
      for (int j = 0; j < st->NE; j++) {
        const int ce = __builtin_popcount(rec[j]);
        for (int b = 0; b < 3; b++)
          if ((ce >> b) & 1) rec[st->NE + 3 + b] |= 1u << j;
      }
    }
  } catch (const std::bad_alloc&) {
    delete st;
    return hp::fail(HP_ENOMEM, "hp_enumerate_structures: out of host memory");
  }
  *out = st;
  return HP_OK;
}

extern "C" int hp_structs_info(const hp_structs* s, int32_t* N, int32_t* S, int32_t* S_dir, int32_t* C) {
  if (!s) return hp::fail(HP_EINVAL, "hp_structs_info: library is NULL");
  if (N) *N = s->N;
  if (S) *S = s->S;
  if (S_dir) *S_dir = s->S_dir;
  if (C) *C = s->C;
  return HP_OK;
}

extern "C" int hp_structs_export(const hp_structs* s, uint8_t* coords, uint8_t* contacts, int32_t* conf_class) {
  if (!s) return hp::fail(HP_EINVAL, "hp_structs_export: library is NULL");
  if (coords) std::memcpy(coords, s->conf.data(), s->conf.size());
  if (contacts && s->C > 0) std::memcpy(contacts, s->contacts.data(), (size_t)s->S_dir * s->C * 2);
  if (conf_class) std::memcpy(conf_class, s->conf_class.data(), sizeof(int32_t) * (size_t)s->S_dir);
  return HP_OK;
}
