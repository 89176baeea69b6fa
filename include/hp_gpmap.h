/*
 * hp_gpmap.h -- C ABI of the GB300 HP-model genotype-phenotype map library.
 *
 * Method: arXiv 2008.05612 (Owen), "GPU accelerated enumeration and
 * exploration of model genotype-phenotype maps for protein folding".
 *
 * Conventions used by every entry point
 *   - A sequence (genotype) of N residues is a 64-bit id g; bit i of g is
 *     residue i, 1 = H (hydrophobic), 0 = P (polar).
 *   - Energies are the Li et al. values of Table 1 scaled by 10 to integers
 *     (Section 2.2): HH = -23, HP = PH = -10, PP = 0, summed over contacts as
 *     in Eq. 1 (lattice neighbours that are not chain neighbours).
 *   - A conformation is a Hamiltonian path of the box (a compact
 *     self-avoiding walk, Section 2.1) modulo the box's rotations and
 *     reflections G; a class (the phenotype) is a conformation modulo G and
 *     chain reversal.  Every conformation competes; a sequence folds to the
 *     class of the unique lowest-energy conformation and otherwise gets the
 *     deleterious phenotype -1 (Section 2.1, energy-threshold paragraph, with
 *     threshold 1 in integer units as in Appendix C).  Where a call takes a
 *     gap_threshold T, a sequence folds iff E2 - E1 >= T, E2 the second-lowest
 *     energy counted with multiplicity; T = 1 is the rule just stated.
 *   - Box sizes: the enumeration time and the library grow quickly with N
 *     (3x3x3: 103,346 conformations in about 0.5 s; 2x4x4: 4.4 million in
 *     about 20 s); the map kernels take boxes with fewer than 65,535 classes.
 *   - Class ids are ranks of class representatives: the representative is
 *     the lexicographically smallest tuple (site(r_0), ..., site(r_{N-1})),
 *     site = x + Lx*(y + Ly*z), over G and both directions.
 *   - Device pointers are plain CUDA device addresses owned by the caller;
 *     `stream` is a cudaStream_t (NULL = legacy default stream).  All work is
 *     stream-ordered.  Calls that check a device-side error word read it back
 *     and therefore SYNCHRONISE their stream before returning: the map calls
 *     (hp_phenotype_map, hp_phenotype_map_batch, hp_autotune), the map
 *     reductions (hp_designability, hp_designability_noalloc,
 *     hp_robustness, hp_neighbourhood, hp_phi_matrix, hp_robustness_cross,
 *     hp_neutral_components), hp_stream_shards, hp_batch_plan_status,
 *     hp_mlp_status, and the network calls that read a value back.  The
 *     others (hp_sequence_scan, hp_sequence_scan_gap, hp_mlp_topk,
 *     hp_mlp_logits, hp_proposal_conformations after its first call,
 *     hp_batch_plan_launch) return as soon as their work is enqueued.  No
 *     call aborts the process; each returns an hp_status and leaves a
 *     message for hp_last_error().
 */
#ifndef HP_GPMAP_H
#define HP_GPMAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HP_OK = 0,
  HP_EINVAL = -1,        /* bad argument (null pointer, size, shape) */
  HP_ENOMEM = -2,        /* host or device allocation failed */
  HP_ECUDA = -3,         /* a CUDA runtime call failed */
  HP_ETIMEOUT = -4,      /* a bounded device-side wait gave up */
  HP_EUNSUPPORTED = -5   /* valid request this build does not implement */
} hp_status;

typedef struct hp_structs hp_structs; /* opaque fold library, library-owned */

/* Enumerate the fold library of a box (Section 2.1: all compact
 * self-avoiding walks), reduced by G and reversal.
 *   ndim: 2 or 3; dims[0..ndim-1]: side lengths (>= 1), N = product <= 40.
 *   out:  receives a new library handle; free it with hp_structs_free.
 * Host-only call.  Fails with HP_EINVAL for bad shapes, HP_EUNSUPPORTED for
 * N > 40, HP_ENOMEM if the library does not fit in host memory. */
int hp_enumerate_structures(int ndim, const int32_t dims[3], hp_structs** out);

/* Sizes of a library: N residues, S classes (phenotypes), S_dir directed
 * conformations (S <= S_dir <= 2S), C contacts per conformation (the same for
 * every compact walk).  Any output pointer may be NULL. */
int hp_structs_info(const hp_structs* s, int32_t* N, int32_t* S, int32_t* S_dir, int32_t* C);

/* Copy the library out to host memory (any pointer may be NULL):
 *   coords:     S_dir x N site indices, conformations in canonical order
 *               (by class, canonical orientation first);
 *   contacts:   S_dir x C x 2 residue indices (i < j) of each contact,
 *               sorted by (i, j);
 *   conf_class: S_dir class ids. */
int hp_structs_export(const hp_structs* s, uint8_t* coords, uint8_t* contacts, int32_t* conf_class);

void hp_structs_free(hp_structs* s);

/* Ground-state phenotype of every sequence id in [seq_begin, seq_begin +
 * seq_count) (Section 2.1; Appendix C kernel semantics).
 *   gap_threshold: minimum energy gap E2 - E1 (x 10 units, E2 the second-
 *                  lowest energy counted with multiplicity) for a sequence to
 *                  fold; 1 = strict uniqueness (the paper's value); values in
 *                  [2, 2^20] run a variant of the map kernel that also keeps
 *                  the second-best tile maximum, always in the default shape
 *                  (reg_bits 5, tile 256); < 1 or > 2^20 give HP_EINVAL.
 *   d_phen:        device int32[seq_count]; d_phen[k] = phenotype of
 *                  seq_begin + k: class id, or -1.
 *   d_argmin_aux:  optional device int32[seq_count] (NULL to skip): class of
 *                  the lowest-index conformation reaching the minimum energy,
 *                  tied or not (training labels for the learned proposal).
 * seq_begin + seq_count must not exceed 2^N.  Allocates a small stream-
 * ordered scratch block (work counter and error word) per call and
 * synchronises `stream` (it reads the error word back: HP_ETIMEOUT when a
 * bounded device wait gave up, see hp_set_wait_limit). */
int hp_phenotype_map(const hp_structs* s, uint64_t seq_begin, uint64_t seq_count, int32_t gap_threshold,
                     int32_t* d_phen, int32_t* d_argmin_aux, void* stream);

/* Kernel shape of the phenotype map: 2^reg_bits sequences per thread (32 =
 * one 32-bit word of sequences per lane at reg_bits 5) and `tile`
 * conformations per shared-memory tile.  Compiled shapes: reg_bits 4 with tile
 * 64 or 128; reg_bits 5 or 6 with tile 64, 128 or 256.  Results never depend
 * on the shape, only speed does.  (No counterpart in the paper, whose kernel
 * had one thread per sequence; Figure 4 sweeps its launch shape instead.) */
typedef struct {
  int32_t reg_bits;
  int32_t tile;
} hp_tile_cfg;

/* Shape used by hp_phenotype_map for this library; NULL restores the default
 * (reg_bits 5, tile 256).  HP_EINVAL for a shape that is not compiled. */
int hp_set_tile_cfg(hp_structs* s, const hp_tile_cfg* cfg);
int hp_get_tile_cfg(const hp_structs* s, hp_tile_cfg* cfg);
/* The compiled shapes: writes up to *n entries to cfgs (may be NULL) and sets
 * *n to the number of shapes. */
int hp_tile_cfg_list(hp_tile_cfg* cfgs, int32_t* n);

/* Autotuner (the analogue of the paper's launch-shape sweep, Section 2.2,
 * Figure 4): times every compiled shape on two waves of work items of this
 * box on the current device, keeps the fastest on the library (as by
 * hp_set_tile_cfg) and returns it in *best (may be NULL).  ms (may be NULL)
 * receives one time per shape in hp_tile_cfg_list order (-1: does not fit).
 * Allocates a stream-ordered scratch map of up to 2^28 ids; synchronises. */
int hp_autotune(hp_structs* s, hp_tile_cfg* best, float* ms, void* stream);

/* Batched persistent launch: the phenotype maps of n boxes (1 <= n <= 8, any
 * shapes and sizes) and their id ranges in ONE launch of the phenotype kernel,
 * whose CTAs take work items from a shared queue (boxes with more
 * conformations first).  Entry i computes exactly what
 * hp_phenotype_map(libs[i], begins[i], counts[i], 1, d_phen[i], NULL) would.
 *   cfg: kernel shape for the launch, NULL for libs[0]'s (see hp_set_tile_cfg).
 * Synchronises `stream` before returning (it reads the error word back). */
int hp_phenotype_map_batch(const hp_structs* const* libs, const uint64_t* begins, const uint64_t* counts, int32_t n,
                           int32_t* const* d_phen, const hp_tile_cfg* cfg, void* stream);

/* The batched launch at an energy-gap threshold (Section 2.1; see
 * hp_phenotype_map): entry i computes exactly what
 * hp_phenotype_map(libs[i], begins[i], counts[i], gap_threshold, d_phen[i],
 * NULL) would.  Thresholds above 1 run all boxes in one launch of the gap
 * variant of the map kernel (its one compiled shape); 1 is
 * hp_phenotype_map_batch with the default shapes.  gap_threshold outside
 * [1, 2^20] gives HP_EINVAL.  Synchronises `stream`. */
int hp_phenotype_map_batch_gap(const hp_structs* const* libs, const uint64_t* begins, const uint64_t* counts,
                               int32_t n, int32_t gap_threshold, int32_t* const* d_phen, void* stream);

/* A batch captured once into a CUDA graph (queue reset + persistent launch).
 * Create uploads the tables and captures on a private stream; launch replays
 * the graph on `stream` without synchronising; status synchronises `stream`
 * and reports a device-side timeout of the replays since the last status.
 * The plan keeps the library handles and output pointers it was made with:
 * they must outlive it.  Plans must not be launched concurrently. */
typedef struct hp_batch_plan hp_batch_plan;
int hp_batch_plan_create(const hp_structs* const* libs, const uint64_t* begins, const uint64_t* counts, int32_t n,
                         int32_t* const* d_phen, const hp_tile_cfg* cfg, void* stream, hp_batch_plan** out);
int hp_batch_plan_launch(hp_batch_plan* plan, void* stream);
int hp_batch_plan_status(hp_batch_plan* plan, void* stream);
void hp_batch_plan_free(hp_batch_plan* plan);

/* Ground state of an arbitrary list of sequence ids (e.g. a seeded sample,
 * the paper's sampling mode of Table 3), one warp per sequence, with optional
 * exact bound pruning seeded by candidate conformations (the learned
 * proposal).  With A_s(h) = sum_i h_i c_i(s) and B the HH-contact count,
 * -E = 10 A + 3 B <= 10 A + 3 min(C, floor(A/2)) (Eq. 1, Table 1 x 10); A
 * depends on a conformation only through its contact-count vector, so the
 * bound is taken once per group of conformations sharing that vector, and a
 * group whose bound is below the best exact score among the candidates is
 * skipped.  Skips are strict, so results equal the full scan's exactly.
 *   d_ids:      device uint64[n] sequence ids (< 2^N);
 *   d_cand:     device int32[n * k] candidate conformation indices (canonical
 *               order, -1 = none) or NULL for the plain full scan;
 *   d_phen:     device int32[n] phenotypes; d_aux: device int32[n] class of
 *               the lowest-index minimum (or NULL);
 *   d_counters: device uint64[2] (or NULL): conformations evaluated exactly
 *               and group bounds evaluated are ADDED to [0] and [1].
 * Stream-ordered; does not synchronise.  No counterpart in the paper beyond
 * its sampled kernel (Appendix C). */
int hp_sequence_scan(const hp_structs* s, const uint64_t* d_ids, int64_t n, const int32_t* d_cand, int32_t k,
                     int32_t* d_phen, int32_t* d_aux, uint64_t* d_counters, void* stream);

/* hp_sequence_scan at an energy-gap threshold, with the gap itself (the
 * Appendix C kernel returns the lowest energy's fold and E1 - E2).  A sequence
 * folds iff E2 - E1 >= gap_threshold (Section 2.1), E2 the second-lowest
 * energy counted with multiplicity (0 gap when the minimum is tied).  Pruning
 * skips a group only when its bound lies gap_threshold or more below the
 * best candidate score, so phenotypes stay exact.
 *   gap_threshold: 1 .. 2^20 (HP_EINVAL otherwise); 1 with d_gap NULL is
 *                  exactly hp_sequence_scan;
 *   d_gap:         device int32[n] or NULL: E2 - E1, INT32_MAX when the box
 *                  has a single conformation; clipped at gap_threshold when
 *                  d_cand is given (pruned conformations are only known to
 *                  lie that far above E1).
 * Other arguments, ownership and errors as hp_sequence_scan. */
int hp_sequence_scan_gap(const hp_structs* s, const uint64_t* d_ids, int64_t n, const int32_t* d_cand, int32_t k,
                         int32_t gap_threshold, int32_t* d_phen, int32_t* d_aux, int32_t* d_gap,
                         uint64_t* d_counters, void* stream);

/* ---- Learned proposal (no counterpart in the paper).  A network
 * N -> H1 -> H2 -> S (ReLU, softmax over the S classes) reads the bits of a
 * sequence id (1 = H) and proposes likely ground-state classes; their
 * conformations seed the exact bound pruning of hp_sequence_scan.  It never
 * decides a phenotype.  Weights are fp32 masters with bf16 copies; every
 * matrix product is a bf16 tensor-core GEMM with fp32 accumulation (tcgen05
 * with a tensor-memory accumulator where the contraction length is a multiple
 * of 64, else mma.sync); training
 * minimises the mean cross-entropy with Adam (beta 0.9 / 0.999, eps 1e-8). */
typedef struct hp_mlp hp_mlp;

/* Create a network on the current device.  H1, H2 multiples of 32; max_batch
 * rows per step.  h_params[0..5] are host fp32 arrays W1 [H1 x N], b1 [H1],
 * W2 [H2 x H1], b2 [H2], W3 [S x H2], b3 [S] (row-major), copied in. */
int hp_mlp_create(int32_t N, int32_t H1, int32_t H2, int32_t S, int32_t max_batch, const float* const* h_params,
                  hp_mlp** out);
void hp_mlp_free(hp_mlp* m);

/* Gradients of the cross-entropy of n (<= max_batch) device ids and class
 * labels without updating: the loss is the sum over rows whose label is not
 * -1, divided by n; h_grads[0..5] (entries may
 * be NULL) receive fp32 gradients in the layout of h_params; *h_loss (may be
 * NULL) the mean loss.  Synchronises `stream` when anything is read back. */
int hp_mlp_gradients(hp_mlp* m, const uint64_t* d_ids, const int32_t* d_labels, int32_t n, float* const* h_grads,
                     float* h_loss, void* stream);

/* One Adam step (Kingma & Ba; b1 0.9, b2 0.999, eps 1e-8, bias-corrected) on
 * n (<= max_batch) ids / labels with learning rate lr; the mean loss before
 * the step goes to *h_loss if non-NULL (synchronises).  The step is the one
 * hp_mlp_gradients' gradients give (the output layer's update is applied
 * inside the GEMM that forms its gradient).  The next hp_mlp_topk refreshes
 * the output layer's class-scattered copy first, on its own stream: order a
 * train step and a top-k on different streams yourself. */
int hp_mlp_train_step(hp_mlp* m, const uint64_t* d_ids, const int32_t* d_labels, int32_t n, float lr, float* h_loss,
                      void* stream);

/* Logits (fp32, n x S row-major, device) of n <= max_batch ids. */
int hp_mlp_logits(hp_mlp* m, const uint64_t* d_ids, int32_t n, float* d_logits, void* stream);

/* The k (1..16) highest-scoring classes of each of n ids (ties toward the
 * lower class), into device int32[n x k]; runs in chunks of max_batch. */
int hp_mlp_topk(hp_mlp* m, const uint64_t* d_ids, int64_t n, int32_t k, int32_t* d_top, void* stream);

/* Drain `stream` and report whether any GEMM of this network since the last
 * check timed out: the tcgen05 GEMM waits on its shared-memory mbarriers with
 * an iteration limit and, when one runs out, records it in a device word of
 * the network and skips its output tile.  Returns HP_OK, HP_ETIMEOUT (results
 * since the last check are invalid; the word is cleared) or HP_ECUDA.
 * hp_mlp_gradients and hp_mlp_train_step check it themselves whenever they
 * synchronise; hp_mlp_logits and hp_mlp_topk are asynchronous and leave it to
 * this call. */
int hp_mlp_status(hp_mlp* m, void* stream);

/* Expand classes (device int32[n x k], -1 allowed) into their conformations:
 * d_cand[n x 2k], entry 2j + q = q-th conformation of class j or -1.
 * n >= 0 and k >= 1 (HP_EINVAL otherwise).  The class tables are built on the
 * device on first use (synchronous upload); the expansion is stream-ordered. */
int hp_proposal_conformations(const hp_structs* s, const int32_t* d_top, int64_t n, int32_t k, int32_t* d_cand,
                              void* stream);

/* Designability (Section 2.3): d_hist[p] = #{k : d_phen[k] = p} for
 * p in [0, S), d_hist[S] = #{k : d_phen[k] = -1}.
 *   d_phen: device int32[count], entries in [-1, S); d_hist: device
 *   uint64[S + 1], overwritten.  Synchronises `stream`: entries outside
 *   [-1, S) are counted nowhere and make the call return HP_EINVAL. */
int hp_designability(const int32_t* d_phen, uint64_t count, int32_t S, uint64_t* d_hist, void* stream);

/* Designability without any device allocation: the same result as
 * hp_designability, for callers that must not have a library allocate device
 * memory -- typically a process whose framework or service already owns the
 * device memory in its own pool, where cudaMalloc/cudaMallocAsync could fail or
 * fragment that pool, or code held to a fixed device-memory budget.  The paper
 * has no counterpart; this is an interface convenience of this library.
 *   Scratch (partial histograms and the error word) is a 4 MiB file-scope
 *   device array that every GPU loading the library holds until exit.
 *   Limit: S + 1 bins must fit one shared-memory histogram and the scratch
 *   (S + 1 <= 58,112 on GB300); larger S returns HP_EINVAL with the limit.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress); make that first call before any stream capture.
 *   All calls share the array: calls that overlap on the GPU (other streams,
 *   other host threads) race and must be serialised by the caller.
 *   Synchronises `stream` before returning (it reads the error word back). */
int hp_designability_noalloc(const int32_t* d_phen, uint64_t count, int32_t S, uint64_t* d_hist, void* stream);

/* Numerators of Eq. 2 for p = q, over a FULL map of 2^N sequences (K = 2, so
 * every genotype has (K-1)L = N single-flip neighbours):
 *   d_neutral[p] = sum over g with P(g) = p of #{i : P(g xor 2^i) = p}
 *   d_to_del[p]  = sum over g with P(g) = p of #{i : P(g xor 2^i) = -1}
 * for p in [0, S); index S stands for the deleterious phenotype.  Robustness
 * rho_p = d_neutral[p] / (N * N_p) and phi_del = d_to_del[p] / (N * N_p).
 *   d_phen: device int32[2^N]; d_neutral, d_to_del: device uint64[S + 1].
 * Takes stream-ordered scratch on `stream` (the error word and 16 replicas of
 * the counters, 256 S bytes; without it the counters are updated directly).
 * Synchronises `stream` (error word: HP_EINVAL for entries outside [-1, S)). */
int hp_robustness(const int32_t* d_phen, int32_t N, int32_t S, uint64_t* d_neutral, uint64_t* d_to_del,
                  void* stream);

/* One row of Eq. 2 over a FULL map of 2^N sequences: for phenotype q (-1
 * allowed) d_row[p] = sum over g with P(g) = q of #{i : P(g xor 2^i) = p},
 * index S for -1; phi_pq = d_row[p] / (N * N_q).  This is the neighbourhood
 * of the top fold analysed in Section 3.2 (Figure 7).
 *   d_phen: device int32[2^N]; d_row: device uint64[S + 1], overwritten.
 * Synchronises `stream`. */
int hp_neighbourhood(const int32_t* d_phen, int32_t N, int32_t S, int32_t q, uint64_t* d_row, void* stream);

/* The whole matrix of Eq. 2 numerators over a FULL map of 2^N sequences
 * (Section 2.3, Eq. 2; the null-model comparison of Eq. 3 and Section 3.2
 * reads it): for every ordered pair of phenotypes (q, p), index S for -1,
 *   M[q][p] = #{(g, i) : P(g) = q, P(g xor 2^i) = p},
 * so phi_pq = M[q][p] / (N N_q), rho_q = M[q][q], phi_del = M[q][S] / (N N_q).
 * Output in compressed rows, only the nonzero entries, columns ascending:
 *   d_row_ptr: device uint64[S + 2]; row q is entries [d_row_ptr[q],
 *              d_row_ptr[q + 1]); d_row_ptr[S + 1] = nnz;
 *   d_col:     device int32[cap] column p of each entry (S for -1);
 *   d_count:   device uint64[cap] M[q][p] of each entry;
 *   *h_nnz:    host; the number of nonzero entries.
 *   d_phen: device int32[2^N], S in [1, 65534], cap in [1, 2^30].
 * When the matrix has more than cap nonzero entries, returns HP_ENOMEM with
 * *h_nnz = the number needed (0 if the count itself overflowed its table of
 * 2 cap slots: retry with a larger cap) and writes no output.  Allocates a
 * stream-ordered scratch block of about 12 x 2 cap + 12 x cap bytes;
 * synchronises `stream` (it reads the entry count back). */
int hp_phi_matrix(const int32_t* d_phen, int32_t N, int32_t S, uint64_t cap, uint64_t* d_row_ptr, int32_t* d_col,
                  uint64_t* d_count, uint64_t* h_nnz, void* stream);

/* Eq. 2 numerators across one high bit between two equally sized aligned
 * blocks: genotype base_a + x of block A flips to base_b + x of block B.
 * ADDS to d_neutral[P_A(x)] when P_B(x) = P_A(x) and to d_to_del[P_A(x)]
 * when P_B(x) = -1 (index S for -1, where both rows count -1 -> -1).
 * Used by the shard streamer for flips between shards.  Synchronises
 * `stream`. */
int hp_robustness_cross(const int32_t* d_phen_a, const int32_t* d_phen_b, uint64_t count, int32_t S,
                        uint64_t* d_neutral, uint64_t* d_to_del, void* stream);

/* Shard streamer (the paper's 6x6 run of 2^36 genotypes, "underway" in
 * Sections 3.1 and 4): the full map of a box computed in 2^shard_bits shards
 * of 2^(N - shard_bits) ids, with designability and the Eq. 2 numerators over
 * ALL N flip directions accumulated exactly (uint64) into host arrays
 * h_hist, h_neutral, h_to_del [S + 1] -- equal to hp_designability and
 * hp_robustness of the full map.  Shard maps live in `window` device buffers
 * of 4 * 2^(N - shard_bits) bytes (window >= 2^(shard_bits-1) + 1, else
 * HP_EINVAL before any device work).  out_dir (NULL: none) receives a
 * manifest and one record per shard and per shard pair, written atomically;
 * a rerun with the same out_dir reuses every record whose table hash matches
 * and computes only the shard maps that missing records need (their number
 * goes to *h_maps_computed if non-NULL).  Synchronises `stream`. */
int hp_stream_shards(const hp_structs* s, int32_t shard_bits, int32_t window, const char* out_dir, uint64_t* h_hist,
                     uint64_t* h_neutral, uint64_t* h_to_del, int32_t* h_maps_computed, void* stream);

/* Neutral networks (Section 1; never computed in the paper): connected
 * components of the graph whose vertices are sequences with P(g) != -1 and
 * whose edges join g and g xor 2^i when P is equal.
 *   d_phen:  device int32[2^N], N <= 31;
 *   d_label: device int32[2^N]; d_label[g] = smallest id in g's component,
 *            -1 where P(g) = -1;
 *   d_ncomp: device uint64[S]; number of components of each phenotype.
 * Synchronises `stream` (HP_ETIMEOUT if a union's bounded retries ran out). */
int hp_neutral_components(const int32_t* d_phen, int32_t N, int32_t S, int32_t* d_label, uint64_t* d_ncomp,
                          void* stream);

/* Neutral-network counts of a space too large for one label array (the 6x6
 * space of 2^36 genotypes, Sections 3.1 and 4; networks as in
 * hp_neutral_components, Section 1): h_ncomp[p] = number of connected
 * components of phenotype p over the whole space [0, 2^N), equal to
 * hp_neutral_components' d_ncomp of the full map where that fits.  The space
 * is cut into 2^shard_bits shards of 2^(N - shard_bits) <= 2^31 ids; each
 * shard's local components come from the union-find of
 * hp_neutral_components over the shard, the flips of the shard bits join them
 * (distinct joins collected per pair of neighbouring shards on the device),
 * and a host union-find merges them.  window: resident shard maps,
 * >= 2^(shard_bits-1) + 1 (HP_EINVAL before any device work otherwise).
 *   h_ncomp: host uint64[S]; *h_maps_computed (may be NULL): shard maps made.
 * Allocates device memory for the window, two label buffers and the join
 * tables; synchronises `stream`. */
int hp_stream_components(const hp_structs* s, int32_t shard_bits, int32_t window, uint64_t* h_ncomp,
                         int32_t* h_maps_computed, void* stream);

/* Thread-local text of the last failure in this library (never NULL). */
const char* hp_last_error(void);

/* Failure-detection hook (no counterpart in the paper).  Every wait of the
 * map kernel and of the tcgen05 GEMM on a shared-memory barrier is bounded:
 * after a number of polls it gives up, the kernel records the timeout in its
 * device error word, stops, waits (with a fixed bound of its own) for the
 * copies and tensor-core operations it still has in flight, and returns, and
 * the call reports HP_ETIMEOUT (hp_phenotype_map, the batch and plan calls,
 * hp_autotune) or hp_mlp_status does.  This call sets the poll limit of those
 * waits for every later launch in the process: polls >= 0 sets it (0 gives
 * up at the first check, which lets a test see the timeout path end in
 * HP_ETIMEOUT with the context still usable), polls < 0 restores each
 * kernel's built-in limit.  The exit drains keep their fixed limit.  It is a
 * process-wide setting for tests: launches made while it is lowered fail.
 * Graph plans keep the limit they were created with.  Always HP_OK. */
int hp_set_wait_limit(int64_t polls);

#ifdef __cplusplus
}
#endif

#endif /* HP_GPMAP_H */
