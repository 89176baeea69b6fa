// The tcgen05 GEMM: C = A B^T for bf16 A [M x K] and B [N x K] (both K-major, row strides a
// multiple of 8 elements, 16-byte aligned bases), fp32 accumulation in tensor memory.
// Either the tile is stored (fp32 and / or bf16, after an optional bias per column and ReLU) or,
// in top-k mode, each row keeps only its kt best (bias-added) columns per 256-column tile.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace hp {

constexpr int kTcTileM = 128, kTcTileN = 256;
constexpr int kTcListsPerTile = 2;  // top-k mode: candidate lists per row and 256-column tile range

struct TcEpilogue {
  const float* bias = nullptr;  // [N] added to every row, or null
  int relu = 0;
  float* Cf = nullptr;  // fp32 output [M x ldcf] or null
  int ldcf = 0;
  __nv_bfloat16* Cb = nullptr;  // bf16 output [M x ldcb] or null
  int ldcb = 0;
  // top-k mode (kt in {4, 8, 16}, outputs ignored): the columns are split into
  // L = tc_topk_lists(M, N) disjoint sets (unions of 128-column slices of the 256-column tiles);
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
  //   kt = -1 (row statistics): per row and column list l (as in top-k mode) the running
  //     maximum m and sum of exp(x - m) go to stats[2 (l M + r) + {0, 1}]; the logit at the row's
  //     label goes to zlab[r];
  //   kt = -2 (cross-entropy gradient): with row_m / row_inv the row's maximum and 1 / sum,
  //     dz = (exp(x - m) / sum - [column == label]) * scale, zero for label -1, stored as bf16 both
  //     row-major (dz, row stride ldz) and transposed (dzt, row stride ldzt)
  const int32_t* labels = nullptr;
  float* stats = nullptr;
  float* zlab = nullptr;
  const float* row_m = nullptr;
  const float* row_inv = nullptr;
  float scale = 1.f;
  __nv_bfloat16* dz = nullptr;
  int ldz = 0;
  __nv_bfloat16* dzt = nullptr;
  int ldzt = 0;
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

// Number of candidate lists per row that top-k mode writes (at most 2 ceil(N / 256)).
int tc_topk_lists(int M, int N);

// Combine the row-statistics lists of kt = -1 mode: row_m[r], row_inv[r] = 1 / sum, and for
// labelled rows log(sum) + m - zlab[r] added to *loss.
void tc_softmax_finish(const float* stats, int lists, int rows, const int32_t* labels, const float* zlab, float* row_m,
                       float* row_inv, float* loss, cudaStream_t st);

// Per row, the k <= kt best of the candidates tc_gemm wrote for `tiles` column lists (ties toward
// the lower index); out[r * k + j], -1 for a missing entry or an index >= S.
void tc_topk_merge(const float* cand_v, const int32_t* cand_i, int tiles, int rows, int kt, int k, int S, int32_t* out,
                   cudaStream_t st);

}  // namespace hp
