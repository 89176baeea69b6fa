// The tcgen05 GEMM: C = A B^T for bf16 A [M x K] and B [N x K], fp32 accumulation in tensor
// memory.  Each operand is K-major (A stored [M][K], B [N][K]) or, with a_mn / b_mn, MN-major
// (A stored [K][M], B [K][N], i.e. the GEMM reads the transpose of a row-major matrix); row
// strides a multiple of 8 elements, 16-byte aligned bases.
// Either the tile is stored (fp32 and / or bf16, after an optional bias per column and ReLU) or,
// in top-k mode, each row keeps only its kt best (bias-added) columns per 256-column tile.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

namespace hp {

// Programmatic dependent launch.  A kernel started by launch_pdl may begin (be scheduled, run its
// set-up) while the kernel before it on the stream is still running; it calls pdl_wait() before
// its first access to global memory, which returns once that kernel has completed and its writes
// are visible, and then pdl_trigger(), which lets the next such kernel be scheduled.  Kernels that
// call them behave as usual under an ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

constexpr int kTcTileM = 128, kTcTileN = 256;
constexpr int kTcStatsListsPerTile = 4;  // row-statistics mode: lists per row and tile range
constexpr int kTcTopkSlotsPerTile = 32;  // top-k mode: candidate slots per row and tile range (lists x kt)
// top-k mode: candidate lists per row and 256-column tile range, one per epilogue warp of a
// tensor-memory lane quarter (two; four, with 16 epilogue warps, measured 4 % slower for k = 4)
__host__ __device__ constexpr int tc_topk_lists_per_tile(int) { return 2; }

struct TcEpilogue {
  bool a_mn = false, b_mn = false;  // operand layouts (see above)
  const float* bias = nullptr;  // [N] added to every row, or null
  int relu = 0;
  float* Cf = nullptr;  // fp32 output [M x ldcf] or null
  int ldcf = 0;
  __nv_bfloat16* Cb = nullptr;  // bf16 output [M x ldcb] or null
  int ldcb = 0;
  // top-k mode (kt in {4, 8, 16}, outputs ignored): the columns are split into
  // L = tc_topk_lists(M, N, kt) disjoint sets (unions of 128-column slices of the 256-column
  // tiles);
  // per row r and set l, the kt largest values with their column indices, sorted (value
  // descending, index ascending), go to cand_v / cand_i [(l * M + r) * kt + j]; missing entries
  // are (-inf, INT32_MAX)
  int kt = 0;
  float* cand_v = nullptr;
  int32_t* cand_i = nullptr;
  // top-k mode: if set, column c is reported (and ordered on ties) as col_id[c] instead of c
  const int32_t* col_id = nullptr;
  // softmax modes over the columns of each row (the proposal's training step; bias added, rows
  // with label -1 ignored):
  //   kt = -1 (row statistics): the columns are split into L = tc_stats_lists(M, N) disjoint
  //     sets (unions of 64-column slices of the tiles); per row r and set l the running maximum m
  //     and sum of exp(x - m) go to stats[2 (l M + r) + {0, 1}]; the logit at the row's label goes
  //     to zlab[r];
  //   kt = -2 (cross-entropy gradient): with row_m / row_inv the row's maximum and 1 / sum and
  //     zlab the label logits of the statistics pass,
  //     dz = (exp(x - m) / sum - [column == label]) * scale, zero for label -1, stored as bf16 both
  //     row-major (dz, row stride ldz >= N, a multiple of 8; base 16-byte aligned; it leaves
  //     through TMA stores, columns >= N and rows >= M are not written); if colpart is set,
  //     colpart[b * N + c] = the sum over the rows
  //     32 b .. 32 b + 31 of the stored (bf16) dz[row, c], in a fixed order
  const int32_t* labels = nullptr;
  float* stats = nullptr;
  float* zlab = nullptr;
  const float* row_m = nullptr;
  const float* row_inv = nullptr;
  float scale = 1.f;
  __nv_bfloat16* dz = nullptr;
  int ldz = 0;
  float* colpart = nullptr;
  // store mode: if set, an element whose activation relu_mask[r * ldmask + c] (bf16) is not
  // positive is stored as 0 (the backward step of a ReLU layer)
  const __nv_bfloat16* relu_mask = nullptr;
  int ldmask = 0;
  // store mode with an Adam step in place of the fp32 store (no bias, ReLU or split-K): the tile
  // is the gradient g of the fp32 weights adam_w [M x ldcf] with moments adam_m, adam_v (same
  // layout); per element m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  // w -= lr (m c1) / (sqrt(v c2) + eps); the new w also goes to Cb (bf16) and, if set, transposed
  // to wt (bf16, wt[c * ldwt + r])
  float* adam_w = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float lr = 0.f, b1 = 0.f, b2 = 0.f, eps = 0.f, c1 = 0.f, c2 = 0.f;
  __nv_bfloat16* wt = nullptr;
  int ldwt = 0;
  // split-K (store mode, fp32 output only, no bias / ReLU): the K chunks are cut into ksplit
  // contiguous slices computed by different CTAs; slice j's partial product goes to
  // Cf + j * split_stride, and the caller sums the slices
  int ksplit = 1;
  size_t split_stride = 0;
};

// Launch on `st`.  A bounded wait that gives up sets *err (device word, may be null) to nonzero
// and leaves that CTA's remaining tiles unwritten.  Returns an HP_* status.
int tc_gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K, const TcEpilogue& ep,
            unsigned* err, cudaStream_t st);

// Number of candidate lists per row that top-k mode writes (at most
// tc_topk_lists_per_tile(kt) ceil(N / 256)).
int tc_topk_lists(int M, int N, int kt);

// Number of statistics lists per row that row-statistics mode writes (at most 4 ceil(N / 256)).
int tc_stats_lists(int M, int N);

// Combine the row-statistics lists of kt = -1 mode: row_m[r], row_inv[r] = 1 / sum, and for
// labelled rows log(sum) + m - zlab[r] added to *loss.
void tc_softmax_finish(const float* stats, int lists, int rows, const int32_t* labels, const float* zlab, float* row_m,
                       float* row_inv, float* loss, cudaStream_t st);

// Per row, the k <= kt best of the candidates tc_gemm wrote for `tiles` column lists (ties toward
// the lower index); out[r * k + j], -1 for a missing entry or an index >= S.
void tc_topk_merge(const float* cand_v, const int32_t* cand_i, int tiles, int rows, int kt, int k, int S, int32_t* out,
                   cudaStream_t st);

}  // namespace hp
