/*
 * hp_oracle.c -- plain, slow CPU oracle for the HP-model genotype-phenotype map.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or generator with the CUDA library; neither includes the other.
 *
 * What it computes (arXiv 2008.05612):
 *   - Section 2.1: the fold library is the set of compact self-avoiding walks,
 *     i.e. Hamiltonian paths of the L x L (x L) box.  Walks are enumerated here
 *     by plain recursive backtracking over lattice coordinates and reduced by
 *     the box's rotation/reflection group G (applied to coordinates) and by
 *     chain reversal.
 *   - Eq. 1: H = sum_{i<j} E(s_i, s_j) Delta(r_i - r_j), Delta = 1 for lattice
 *     neighbours that are not chain neighbours.  Energies are Table 1 scaled by
 *     10 (Section 2.2): HH = -23, HP = PH = -10, PP = 0.  Bit i of the sequence
 *     id is residue i, 1 = H.
 *   - Section 2.1 (last paragraph): a sequence folds to the lowest-energy fold
 *     if the gap to the second-lowest energy is at least the threshold
 *     (threshold 1 in integer units = strict uniqueness); otherwise it has the
 *     deleterious phenotype (-1).
 *   - Section 2.3: designability N_q (count of genotypes per phenotype), the
 *     single-point-mutation neighbourhood (K-1)L = N for K = 2, Eq. 2
 *     (phi_pq) and robustness rho_p = phi_pp; phi_del counts flips into -1.
 *   - Neutral networks (Section 1): connected components of the graph of
 *     genotypes joined by neutral single flips, labelled by their smallest id.
 *
 * Readings taken where the paper is silent (each listed in the design notes):
 *   reading B (default): every directed conformation (a Hamiltonian path modulo
 *     G, reversal NOT applied) competes; a tie between two distinct
 *     conformations -- even the two orientations of one class -- is not unique.
 *     The phenotype is the class (conformation modulo G and reversal).
 *   reading A: only the canonical orientation of each class competes.
 *   reading C: all conformations compete, uniqueness is judged per class.
 *   Class id = rank of the class representative, the lexicographically
 *   smallest site tuple (site = x + Lx*(y + Ly*z)) over G and both directions.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXN 64
#define OR_MAXG 48

typedef struct {
  int ndim, L[3], N, nsym;
  int img[OR_MAXG][OR_MAXN];     /* image of each site under each group element */
  int64_t n_paths;               /* raw directed Hamiltonian paths */
  int64_t fix_rev;               /* sum over g of #{p : g(p) == reverse(p)} */
  int32_t S_dir, S, C;
  uint8_t *conf;                 /* S_dir x N sites, sorted by (class rep, tuple) */
  int32_t *conf_class;           /* S_dir */
  uint8_t *contacts;             /* S_dir x C x 2 residue indices, i < j */
  int32_t *contact_count;        /* S_dir: contacts found per conformation */
} or_box;

/* ------------------------------------------------------------------ geometry */

static void site_xyz(const or_box *b, int s, int c[3]) {
  c[0] = s % b->L[0];
  c[1] = (s / b->L[0]) % b->L[1];
  c[2] = s / (b->L[0] * b->L[1]);
}

static int xyz_site(const or_box *b, const int c[3]) {
  return c[0] + b->L[0] * (c[1] + b->L[1] * c[2]);
}

static int adjacent(const or_box *b, int s, int t) {
  int a[3], c[3];
  site_xyz(b, s, a);
  site_xyz(b, t, c);
  int d = abs(a[0] - c[0]) + abs(a[1] - c[1]) + abs(a[2] - c[2]);
  return d == 1;
}

/* The symmetry group of the box: every permutation of the first ndim axes that
 * maps each axis onto one of equal length, combined with every set of
 * reflections. */
static void build_group(or_box *b) {
  static const int perms3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  int n = 0;
  for (int pi = 0; pi < 6; pi++) {
    const int *p = perms3[pi];
    int ok = 1;
    for (int k = 0; k < 3; k++) {
      if (k >= b->ndim && p[k] != k) ok = 0;
      if (b->L[k] != b->L[p[k]]) ok = 0;
    }
    if (!ok) continue;
    for (int fl = 0; fl < (1 << b->ndim); fl++) {
      for (int s = 0; s < b->N; s++) {
        int c[3], d[3];
        site_xyz(b, s, c);
        for (int k = 0; k < 3; k++) {
          int v = c[p[k]];
          if (k < b->ndim && ((fl >> k) & 1)) v = b->L[k] - 1 - v;
          d[k] = v;
        }
        b->img[n][s] = xyz_site(b, d);
      }
      n++;
    }
  }
  b->nsym = n;
  /* element 0 is the identity (first permutation, no reflection) */
}

/* lexicographic comparison of two site tuples */
static int tuple_cmp(const uint8_t *a, const uint8_t *c, int n) {
  for (int i = 0; i < n; i++)
    if (a[i] != c[i]) return a[i] < c[i] ? -1 : 1;
  return 0;
}

/* smallest image of path p under G, written to out */
static void canon(const or_box *b, const uint8_t *p, uint8_t *out) {
  uint8_t t[OR_MAXN];
  memcpy(out, p, b->N);
  for (int g = 0; g < b->nsym; g++) {
    for (int i = 0; i < b->N; i++) t[i] = (uint8_t)b->img[g][p[i]];
    if (tuple_cmp(t, out, b->N) < 0) memcpy(out, t, b->N);
  }
}

/* ------------------------------------------------------------- enumeration */

typedef struct {
  or_box *b;
  int nbr[OR_MAXN][6], nnbr[OR_MAXN]; /* lattice neighbours of each site */
  uint8_t path[OR_MAXN];
  uint8_t visited[OR_MAXN];
  uint8_t *store;
  int64_t cap, count;
} enum_ctx;

static void record_path(enum_ctx *e) {
  or_box *b = e->b;
  int N = b->N;
  b->n_paths++;
  /* fixed points of (g, reversal): g(p) == reverse(p) */
  for (int g = 0; g < b->nsym; g++) {
    int same = 1;
    for (int i = 0; i < N && same; i++)
      if (b->img[g][e->path[i]] != e->path[N - 1 - i]) same = 0;
    b->fix_rev += same;
  }
  /* keep p only if no image g(p) is lexicographically smaller than p */
  for (int g = 1; g < b->nsym; g++) {
    for (int i = 0; i < N; i++) {
      int gi = b->img[g][e->path[i]];
      if (gi < e->path[i]) return;
      if (gi > e->path[i]) break;
    }
  }
  if (e->count == e->cap) {
    e->cap = e->cap ? 2 * e->cap : 1024;
    e->store = (uint8_t *)realloc(e->store, (size_t)e->cap * N);
  }
  memcpy(e->store + (size_t)e->count * N, e->path, N);
  e->count++;
}

static void walk(enum_ctx *e, int depth, int site) {
  or_box *b = e->b;
  e->path[depth] = (uint8_t)site;
  e->visited[site] = 1;
  if (depth == b->N - 1) {
    record_path(e);
  } else {
    for (int k = 0; k < e->nnbr[site]; k++) {
      int t = e->nbr[site][k];
      if (!e->visited[t]) walk(e, depth + 1, t);
    }
  }
  e->visited[site] = 0;
}

/* sort key record for ordering conformations by (class rep, own tuple) */
static int g_sortN;
typedef struct {
  uint8_t rep[OR_MAXN];
  uint8_t own[OR_MAXN];
} conf_key;

static int key_cmp(const void *x, const void *y) {
  const conf_key *a = (const conf_key *)x, *c = (const conf_key *)y;
  int r = tuple_cmp(a->rep, c->rep, g_sortN);
  if (r) return r;
  return tuple_cmp(a->own, c->own, g_sortN);
}

/* Enumerate the fold library of an ndim-dimensional box with side lengths
 * dims[0..ndim-1].  Returns NULL on bad arguments. */
or_box *or_enumerate(int ndim, const int32_t *dims) {
  if (ndim != 2 && ndim != 3) return NULL;
  or_box *b = (or_box *)calloc(1, sizeof(or_box));
  b->ndim = ndim;
  b->L[0] = dims[0];
  b->L[1] = dims[1];
  b->L[2] = ndim == 3 ? dims[2] : 1;
  for (int k = 0; k < 3; k++)
    if (b->L[k] < 1) { free(b); return NULL; }
  b->N = b->L[0] * b->L[1] * b->L[2];
  if (b->N < 2 || b->N > OR_MAXN) { free(b); return NULL; }
  build_group(b);

  enum_ctx e;
  memset(&e, 0, sizeof(e));
  e.b = b;
  for (int s = 0; s < b->N; s++) {
    int c[3];
    site_xyz(b, s, c);
    for (int k = 0; k < b->ndim; k++)
      for (int dir = -1; dir <= 1; dir += 2) {
        int d[3] = {c[0], c[1], c[2]};
        d[k] += dir;
        if (d[k] < 0 || d[k] >= b->L[k]) continue;
        e.nbr[s][e.nnbr[s]++] = xyz_site(b, d);
      }
  }
  for (int s = 0; s < b->N; s++) walk(&e, 0, s);

  int N = b->N;
  b->S_dir = (int32_t)e.count;
  conf_key *keys = (conf_key *)calloc((size_t)e.count, sizeof(conf_key));
  for (int64_t i = 0; i < e.count; i++) {
    uint8_t *p = e.store + (size_t)i * N;
    uint8_t r[OR_MAXN], q[OR_MAXN];
    for (int k = 0; k < N; k++) r[k] = p[N - 1 - k];
    canon(b, r, q);
    memcpy(keys[i].own, p, N);
    memcpy(keys[i].rep, tuple_cmp(p, q, N) <= 0 ? p : q, N);
  }
  g_sortN = N;
  qsort(keys, (size_t)e.count, sizeof(conf_key), key_cmp);

  b->conf = (uint8_t *)malloc((size_t)e.count * N);
  b->conf_class = (int32_t *)malloc(sizeof(int32_t) * (size_t)(e.count ? e.count : 1));
  int32_t cls = -1;
  for (int64_t i = 0; i < e.count; i++) {
    if (i == 0 || tuple_cmp(keys[i].rep, keys[i - 1].rep, N) != 0) cls++;
    b->conf_class[i] = cls;
    memcpy(b->conf + (size_t)i * N, keys[i].own, N);
  }
  b->S = cls + 1;
  free(keys);
  free(e.store);

  /* contacts: residue pairs i < j, j > i + 1, on lattice-neighbouring sites */
  int maxc = 0;
  b->contact_count = (int32_t *)calloc((size_t)(b->S_dir ? b->S_dir : 1), sizeof(int32_t));
  for (int32_t s = 0; s < b->S_dir; s++) {
    const uint8_t *p = b->conf + (size_t)s * N;
    int c = 0;
    for (int i = 0; i < N; i++)
      for (int j = i + 2; j < N; j++)
        if (adjacent(b, p[i], p[j])) c++;
    b->contact_count[s] = c;
    if (c > maxc) maxc = c;
  }
  b->C = maxc;
  b->contacts = (uint8_t *)calloc((size_t)(b->S_dir ? b->S_dir : 1) * (maxc ? maxc : 1) * 2, 1);
  for (int32_t s = 0; s < b->S_dir; s++) {
    const uint8_t *p = b->conf + (size_t)s * N;
    uint8_t *out = b->contacts + (size_t)s * maxc * 2;
    int c = 0;
    for (int i = 0; i < N; i++)
      for (int j = i + 2; j < N; j++)
        if (adjacent(b, p[i], p[j])) {
          out[2 * c] = (uint8_t)i;
          out[2 * c + 1] = (uint8_t)j;
          c++;
        }
  }
  return b;
}

void or_free(or_box *b) {
  if (!b) return;
  free(b->conf);
  free(b->conf_class);
  free(b->contacts);
  free(b->contact_count);
  free(b);
}

/* info[0..7] = N, S, S_dir, C, nsym, n_paths (low 32), n_paths (high 32), ndim */
void or_info(const or_box *b, int64_t *info) {
  info[0] = b->N;
  info[1] = b->S;
  info[2] = b->S_dir;
  info[3] = b->C;
  info[4] = b->nsym;
  info[5] = b->n_paths;
  info[6] = b->fix_rev;
  info[7] = b->ndim;
}

/* coords: S_dir x N site indices; conf_class: S_dir; contacts: S_dir x C x 2;
 * contact_count: S_dir.  Any pointer may be NULL. */
void or_export(const or_box *b, uint8_t *coords, int32_t *conf_class, uint8_t *contacts, int32_t *contact_count) {
  if (coords) memcpy(coords, b->conf, (size_t)b->S_dir * b->N);
  if (conf_class) memcpy(conf_class, b->conf_class, sizeof(int32_t) * (size_t)b->S_dir);
  if (contacts) memcpy(contacts, b->contacts, (size_t)b->S_dir * b->C * 2);
  if (contact_count) memcpy(contact_count, b->contact_count, sizeof(int32_t) * (size_t)b->S_dir);
}

/* site tuple of the representative of every class (S x N) */
void or_class_reps(const or_box *b, uint8_t *reps) {
  for (int32_t s = 0; s < b->S_dir; s++)
    if (s == 0 || b->conf_class[s] != b->conf_class[s - 1])
      memcpy(reps + (size_t)b->conf_class[s] * b->N, b->conf + (size_t)s * b->N, b->N);
}

/* ----------------------------------------------------------------- energies */

/* Table 1 x 10, indexed [h_i][h_j] with 1 = H */
static const int E_TAB[2][2] = {{0, -10}, {-10, -23}};

/* Eq. 1 for sequence g on conformation s, as a sum over the contact pairs */
int or_energy(const or_box *b, uint64_t g, int32_t s) {
  const uint8_t *c = b->contacts + (size_t)s * b->C * 2;
  int e = 0;
  for (int k = 0; k < b->contact_count[s]; k++) {
    int hi = (int)((g >> c[2 * k]) & 1), hj = (int)((g >> c[2 * k + 1]) & 1);
    e += E_TAB[hi][hj];
  }
  return e;
}

/* Eq. 1 evaluated straight from coordinates: every residue pair i < j that is
 * not bonded and sits on neighbouring lattice sites. */
int or_energy_coords(const or_box *b, uint64_t g, int32_t s) {
  const uint8_t *p = b->conf + (size_t)s * b->N;
  int e = 0;
  for (int i = 0; i < b->N; i++)
    for (int j = i + 1; j < b->N; j++) {
      if (j == i + 1) continue;
      if (!adjacent(b, p[i], p[j])) continue;
      e += E_TAB[(g >> i) & 1][(g >> j) & 1];
    }
  return e;
}

/* The bound used to skip conformations safely: with A = sum_i h_i c_i(s) and
 * B = number of HH contacts, E = -10 A - 3 B, B <= C and 2B <= A, so
 * E >= -10 A - 3 min(C, floor(A/2)). */
int or_lower_bound(const or_box *b, uint64_t g, int32_t s) {
  const uint8_t *c = b->contacts + (size_t)s * b->C * 2;
  int A = 0;
  for (int k = 0; k < b->contact_count[s]; k++) A += (int)((g >> c[2 * k]) & 1) + (int)((g >> c[2 * k + 1]) & 1);
  int Bmax = A / 2 < b->contact_count[s] ? A / 2 : b->contact_count[s];
  return -10 * A - 3 * Bmax;
}

/* ground state of one sequence under the chosen reading; *gap_out (optional)
 * receives e2 - e1, the energy difference the Appendix C kernel returns with
 * its sign flipped, or INT32_MAX when there is a single competitor */
static void ground_state(const or_box *b, uint64_t g, int reading, int gap, int32_t *phen, int32_t *aux,
                         int32_t *gap_out) {
  int e1 = 1 << 30, e2 = 1 << 30;   /* lowest and second-lowest (with multiplicity) */
  int32_t first = -1;               /* lowest-index conformation at e1 */
  int e2_other = 1 << 30;           /* reading C: lowest energy of any other class */
  for (int32_t s = 0; s < b->S_dir; s++) {
    if (reading == 0 && s > 0 && b->conf_class[s] == b->conf_class[s - 1]) continue; /* A: reps only */
    int e = or_energy(b, g, s);
    if (e < e1) {
      e2 = e1;
      e1 = e;
      first = s;
    } else if (e < e2) {
      e2 = e;
    }
  }
  if (reading == 2) {
    /* C: second-lowest energy over conformations of classes other than first's */
    int32_t c1 = b->conf_class[first];
    for (int32_t s = 0; s < b->S_dir; s++) {
      if (b->conf_class[s] == c1) continue;
      int e = or_energy(b, g, s);
      if (e < e2_other) e2_other = e;
    }
    e2 = e2_other;
  }
  int32_t cls = b->conf_class[first];
  if (aux) *aux = cls;
  if (b->S_dir == 1 || (reading == 2 && b->S == 1)) {
    *phen = cls; /* a single competitor is always the unique minimum */
    if (gap_out) *gap_out = INT32_MAX;
    return;
  }
  if (gap_out) *gap_out = e2 - e1;
  *phen = (e2 - e1 >= gap) ? cls : -1;
}

typedef struct {
  const or_box *b;
  const uint64_t *seqs;
  int64_t lo, hi;
  int reading, gap;
  int32_t *phen, *aux, *gaps;
} gs_job;

static void *gs_worker(void *arg) {
  gs_job *j = (gs_job *)arg;
  for (int64_t i = j->lo; i < j->hi; i++)
    ground_state(j->b, j->seqs[i], j->reading, j->gap, &j->phen[i], j->aux ? &j->aux[i] : NULL,
                 j->gaps ? &j->gaps[i] : NULL);
  return NULL;
}

/* Phenotype of each listed sequence id.  reading: 0 = A, 1 = B, 2 = C.
 * aux (optional) receives the class of the lowest-index conformation at the
 * minimum energy, tied or not; gaps (optional) the difference between the
 * second-lowest energy (with multiplicity: 0 when the minimum is tied) and
 * the lowest, INT32_MAX for a single competitor. */
int or_phenotypes_gaps(const or_box *b, const uint64_t *seqs, int64_t n, int reading, int gap, int32_t *phen,
                       int32_t *aux, int32_t *gaps, int nthreads) {
  if (reading < 0 || reading > 2 || gap < 1 || b->S_dir < 1) return -1;
  for (int64_t i = 0; i < n; i++)
    if (b->N < 64 && (seqs[i] >> b->N) != 0) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  gs_job jobs[256];
  for (int t = 0; t < nthreads; t++) {
    jobs[t].b = b;
    jobs[t].seqs = seqs;
    jobs[t].lo = n * t / nthreads;
    jobs[t].hi = n * (t + 1) / nthreads;
    jobs[t].reading = reading;
    jobs[t].gap = gap;
    jobs[t].phen = phen;
    jobs[t].aux = aux;
    jobs[t].gaps = gaps;
    pthread_create(&th[t], NULL, gs_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
  return 0;
}

int or_phenotypes(const or_box *b, const uint64_t *seqs, int64_t n, int reading, int gap, int32_t *phen,
                  int32_t *aux, int nthreads) {
  return or_phenotypes_gaps(b, seqs, n, reading, gap, phen, aux, NULL, nthreads);
}

/* --------------------------------------------------------------- reductions */

static int64_t bucket(int32_t p, int32_t S) { return p < 0 ? S : p; }

/* designability: hist[p] = #{g : P(g) = p}, hist[S] = #{g : P(g) = -1} */
void or_designability(const int32_t *phen, uint64_t count, int32_t S, uint64_t *hist) {
  memset(hist, 0, sizeof(uint64_t) * (size_t)(S + 1));
  for (uint64_t g = 0; g < count; g++) hist[bucket(phen[g], S)]++;
}

/* Eq. 2 numerators over a full map of 2^N genotypes:
 * neutral[p] = sum over g with P(g) = p of #{i : P(g ^ 2^i) = p},
 * to_del[p]  = sum over g with P(g) = p of #{i : P(g ^ 2^i) = -1};
 * index S stands for the deleterious phenotype. */
void or_robustness(const int32_t *phen, int N, int32_t S, uint64_t *neutral, uint64_t *to_del) {
  memset(neutral, 0, sizeof(uint64_t) * (size_t)(S + 1));
  memset(to_del, 0, sizeof(uint64_t) * (size_t)(S + 1));
  uint64_t total = 1ull << N;
  for (uint64_t g = 0; g < total; g++) {
    int32_t p = phen[g];
    for (int i = 0; i < N; i++) {
      int32_t q = phen[g ^ (1ull << i)];
      if (q == p) neutral[bucket(p, S)]++;
      if (q < 0) to_del[bucket(p, S)]++;
    }
  }
}

/* sparse phi_pq numerators for one phenotype q: out[p] = sum over g with
 * P(g) = q of #{i : P(g ^ 2^i) = p}, index S for -1 */
void or_neighbourhood(const int32_t *phen, int N, int32_t S, int32_t q, uint64_t *out) {
  memset(out, 0, sizeof(uint64_t) * (size_t)(S + 1));
  uint64_t total = 1ull << N;
  for (uint64_t g = 0; g < total; g++) {
    if (phen[g] != q) continue;
    for (int i = 0; i < N; i++) out[bucket(phen[g ^ (1ull << i)], S)]++;
  }
}

static uint32_t uf_find(uint32_t *par, uint32_t x) {
  uint32_t r = x;
  while (par[r] != r) r = par[r];
  while (par[x] != r) {
    uint32_t n = par[x];
    par[x] = r;
    x = n;
  }
  return r;
}

/* Neutral components: genotypes with P(g) != -1 joined by single flips that
 * keep the phenotype.  label[g] = smallest id in g's component (-1 for
 * deleterious genotypes); ncomp[p] = number of components of phenotype p. */
int or_components(const int32_t *phen, int N, int32_t S, int32_t *label, uint64_t *ncomp) {
  if (N > 31) return -1;
  uint32_t total = 1u << N;
  uint32_t *par = (uint32_t *)malloc(sizeof(uint32_t) * total);
  if (!par) return -1;
  for (uint32_t g = 0; g < total; g++) par[g] = g;
  for (uint32_t g = 0; g < total; g++) {
    if (phen[g] < 0) continue;
    for (int i = 0; i < N; i++) {
      uint32_t h = g ^ (1u << i);
      if (h < g || phen[h] != phen[g]) continue;
      uint32_t a = uf_find(par, g), c = uf_find(par, h);
      if (a != c) {
        if (a < c) par[c] = a; else par[a] = c;   /* the root is the smaller id */
      }
    }
  }
  memset(ncomp, 0, sizeof(uint64_t) * (size_t)S);
  for (uint32_t g = 0; g < total; g++) {
    if (phen[g] < 0) {
      label[g] = -1;
      continue;
    }
    uint32_t r = uf_find(par, g);
    label[g] = (int32_t)r;
    if (r == g) ncomp[phen[g]]++;
  }
  free(par);
  return 0;
}
