// The learned proposal: an N -> H1 -> H2 -> S network (ReLU, softmax over the
// S classes) on the bits of a sequence id, trained on phenotype maps that the
// exhaustive kernel computes, whose top-k classes seed the bound-pruned scan.
// The paper has no learned component; this only ever proposes candidates, it
// never decides a phenotype.
//
// Kernels (all hand-written): the GEMMs C = A B^T run on the tcgen05 kernel of
// tc_gemm.cu (the output layer of the proposal with its top-k fused into the
// epilogue); the earlier mma.sync m16n8k16 kernels (ldmatrix, cp.async double
// buffering, fused bias / ReLU epilogue) stay as a comparison path selected by
// HP_MLP_LEGACY_MMA=1.  Also here: tiled bf16 transposes, softmax
// cross-entropy, column sums, ReLU backward, Adam, id -> bit encoding and the
// per-row top-k of the comparison path.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "hp_internal.h"
#include "tc_gemm.h"

namespace {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------ GEMM

constexpr int BM = 128, BN = 128, BK = 32, SK = 40;  // SK: padded smem row (elements), 80 B

struct Gemm {
  const bf16* A;  // [M, K] row-major, row stride lda (elements, multiple of 8)
  const bf16* B;  // [N, K] row-major, row stride ldb
  int lda, ldb, M, N, K;  // K a multiple of 32
  const float* bias;      // [N] or NULL
  int relu;
  float* Cf;  // [M, N] fp32 (row stride ldcf) or NULL
  int ldcf;
  bf16* Cb;   // [M, N] bf16 (row stride ldcb) or NULL
  int ldcb;
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"((uint32_t)__cvta_generic_to_shared(p)));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(256) gemm_tn(const Gemm g) {
  __shared__ __align__(16) bf16 sA[2][BM * SK];
  __shared__ __align__(16) bf16 sB[2][BN * SK];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;  // warp tile: 64 rows x 32 columns
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[i][j][q] = 0.f;

  auto load = [&](int stage, int k0) {
#pragma unroll
    for (int i = 0; i < 2; i++) {
      const int c = tid + i * 256, row = c >> 2, kc = (c & 3) * 8;
      const int gr = m0 + row, gn = n0 + row;
      const bf16* pa = gr < g.M ? g.A + (size_t)gr * g.lda + k0 + kc : g.A;
      const bf16* pb = gn < g.N ? g.B + (size_t)gn * g.ldb + k0 + kc : g.B;
      cp_async16(&sA[stage][row * SK + kc], pa, gr < g.M ? 16 : 0);
      cp_async16(&sB[stage][row * SK + kc], pb, gn < g.N ? 16 : 0);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  const int nk = g.K / BK;
  load(0, 0);
  for (int kt = 0; kt < nk; kt++) {
    if (kt + 1 < nk) {
      load((kt + 1) & 1, (kt + 1) * BK);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const bf16* a_s = sA[kt & 1];
    const bf16* b_s = sB[kt & 1];
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[4][4], bfr[2][4];
#pragma unroll
      for (int mi = 0; mi < 4; mi++)
        ldsm_x4(af[mi], a_s + (wm * 64 + mi * 16 + (lane & 15)) * SK + kk + (lane >> 4) * 8);
#pragma unroll
      for (int nj = 0; nj < 2; nj++)
        ldsm_x4(bfr[nj], b_s + (wn * 32 + nj * 16 + (lane >> 4) * 8 + (lane & 7)) * SK + kk + ((lane >> 3) & 1) * 8);
#pragma unroll
      for (int mi = 0; mi < 4; mi++)
#pragma unroll
        for (int ni = 0; ni < 4; ni++) mma_bf16(acc[mi][ni], af[mi], bfr[ni >> 1][(ni & 1) * 2], bfr[ni >> 1][(ni & 1) * 2 + 1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 4; mi++)
#pragma unroll
    for (int ni = 0; ni < 4; ni++) {
      const int col = n0 + wn * 32 + ni * 8 + (lane & 3) * 2;
#pragma unroll
      for (int hrow = 0; hrow < 2; hrow++) {
        const int row = m0 + wm * 64 + mi * 16 + (lane >> 2) + hrow * 8;
        if (row >= g.M) continue;
#pragma unroll
        for (int q = 0; q < 2; q++) {
          const int c = col + q;
          if (c >= g.N) continue;
          float v = acc[mi][ni][hrow * 2 + q];
          if (g.bias) v += g.bias[c];
          if (g.relu) v = fmaxf(v, 0.f);
          if (g.Cf) g.Cf[(size_t)row * g.ldcf + c] = v;
          if (g.Cb) g.Cb[(size_t)row * g.ldcb + c] = __float2bfloat16(v);
        }
      }
    }
}

// Large-tile variant for the big products (the 512 x S output layer): BMxBN CTA tile, BK = 64,
// STAGES-deep cp.async pipeline in dynamic shared memory, 8 warps of 64 x (BN/4) each.
template <int BM_, int BN_, int STAGES>
struct BigGemm {
  static constexpr int BM = BM_, BN = BN_, BK = 64, SKB = BK + 8;  // padded row: 144 B (conflict-free ldmatrix)
  static constexpr int WM = 64, WN = BN / 4;                          // 2 x 4 warps
  static constexpr int MI = WM / 16, NI = WN / 8;
  static constexpr size_t kStageElems = (size_t)(BM + BN) * SKB;
  static constexpr size_t kSmemBytes = kStageElems * STAGES * sizeof(bf16);
};

template <int BM_, int BN_, int STAGES>
__global__ void __launch_bounds__(256, 1) gemm_tn_big(const Gemm g) {
  using C = BigGemm<BM_, BN_, STAGES>;
  constexpr int BM = C::BM, BN = C::BN, BK = C::BK, SKB = C::SKB, MI = C::MI, NI = C::NI;
  extern __shared__ __align__(16) bf16 smem_g[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[MI][NI][4];
#pragma unroll
  for (int i = 0; i < MI; i++)
#pragma unroll
    for (int j = 0; j < NI; j++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[i][j][q] = 0.f;
  auto sa = [&](int st) { return smem_g + (size_t)st * C::kStageElems; };
  auto sb = [&](int st) { return smem_g + (size_t)st * C::kStageElems + (size_t)BM * SKB; };
  auto load = [&](int st, int k0) {
    bf16* a_s = sa(st);
    bf16* b_s = sb(st);
    // BK = 64 elements = 8 chunks of 16 B per row
    for (int c = tid; c < BM * 8; c += 256) {
      const int row = c >> 3, kc = (c & 7) * 8, gr = m0 + row;
      cp_async16(a_s + row * SKB + kc, gr < g.M ? g.A + (size_t)gr * g.lda + k0 + kc : g.A, gr < g.M ? 16 : 0);
    }
    for (int c = tid; c < BN * 8; c += 256) {
      const int row = c >> 3, kc = (c & 7) * 8, gn = n0 + row;
      cp_async16(b_s + row * SKB + kc, gn < g.N ? g.B + (size_t)gn * g.ldb + k0 + kc : g.B, gn < g.N ? 16 : 0);
    }
  };
  const int nk = g.K / BK;
#pragma unroll
  for (int st = 0; st < STAGES - 1; st++) {
    if (st < nk) load(st, st * BK);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int kt = 0; kt < nk; kt++) {
    asm volatile("cp.async.wait_group %0;" ::"n"(STAGES - 2) : "memory");
    __syncthreads();
    {
      const int nxt = kt + STAGES - 1;
      if (nxt < nk) load(nxt % STAGES, nxt * BK);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const bf16* a_s = sa(kt % STAGES);
    const bf16* b_s = sb(kt % STAGES);
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[MI][4], bfr[NI / 2][4];
#pragma unroll
      for (int mi = 0; mi < MI; mi++)
        ldsm_x4(af[mi], a_s + (wm * 64 + mi * 16 + (lane & 15)) * SKB + kk + (lane >> 4) * 8);
#pragma unroll
      for (int nj = 0; nj < NI / 2; nj++)
        ldsm_x4(bfr[nj], b_s + (wn * C::WN + nj * 16 + (lane >> 4) * 8 + (lane & 7)) * SKB + kk + ((lane >> 3) & 1) * 8);
#pragma unroll
      for (int mi = 0; mi < MI; mi++)
#pragma unroll
        for (int ni = 0; ni < NI; ni++)
          mma_bf16(acc[mi][ni], af[mi], bfr[ni >> 1][(ni & 1) * 2], bfr[ni >> 1][(ni & 1) * 2 + 1]);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
  for (int mi = 0; mi < MI; mi++)
#pragma unroll
    for (int ni = 0; ni < NI; ni++) {
      const int col = n0 + wn * C::WN + ni * 8 + (lane & 3) * 2;
#pragma unroll
      for (int hrow = 0; hrow < 2; hrow++) {
        const int row = m0 + wm * 64 + mi * 16 + (lane >> 2) + hrow * 8;
        if (row >= g.M) continue;
#pragma unroll
        for (int q = 0; q < 2; q++) {
          const int c = col + q;
          if (c >= g.N) continue;
          float v = acc[mi][ni][hrow * 2 + q];
          if (g.bias) v += g.bias[c];
          if (g.relu) v = fmaxf(v, 0.f);
          if (g.Cf) g.Cf[(size_t)row * g.ldcf + c] = v;
          if (g.Cb) g.Cb[(size_t)row * g.ldcb + c] = __float2bfloat16(v);
        }
      }
    }
}

// ------------------------------------------------------------------ small kernels

// out[c, r] = in[r, c] for r < rows, c < cols; zero in [rows, out_cols) of each output row.
// 64 x 64 tiles; reads and writes move bf16 pairs (4 bytes), so a warp touches 128 contiguous
// bytes of a row on both sides.
__global__ void transpose_bf16(const bf16* __restrict__ in, int ldin, int rows, int cols, bf16* __restrict__ out,
                               int ldout, int out_cols) {
  __shared__ bf16 tile[64][66];
  const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int j = ty; j < 64; j += 8) {
    const int r = r0 + j, c = c0 + 2 * tx;
    bf16 a = __float2bfloat16(0.f), b = a;
    if (r < rows) {
      if (c + 1 < cols && ((ldin | c) & 1) == 0) {
        const __nv_bfloat162 q = *reinterpret_cast<const __nv_bfloat162*>(in + (size_t)r * ldin + c);
        a = q.x;
        b = q.y;
      } else {
        if (c < cols) a = in[(size_t)r * ldin + c];
        if (c + 1 < cols) b = in[(size_t)r * ldin + c + 1];
      }
    }
    tile[j][2 * tx] = a;
    tile[j][2 * tx + 1] = b;
  }
  __syncthreads();
  for (int j = ty; j < 64; j += 8) {
    const int c = c0 + j, r = r0 + 2 * tx;
    if (c >= cols) continue;
    const bf16 a = tile[2 * tx][j], b = tile[2 * tx + 1][j];
    bf16* o = out + (size_t)c * ldout + r;
    if (r + 1 < out_cols && ((ldout | r) & 1) == 0) {
      __nv_bfloat162 q;
      q.x = a;
      q.y = b;
      *reinterpret_cast<__nv_bfloat162*>(o) = q;
    } else {
      if (r < out_cols) o[0] = a;
      if (r + 1 < out_cols) o[1] = b;
    }
  }
}

__global__ void cast_bf16(const float* __restrict__ in, bf16* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16(in[i]);
}

// X[b, i] = bit i of ids[b] (1 = H) for i < N, 0 for i in [N, Kin) and for rows b >= n; with
// lab_out set, also lab_out[b] = lab_in[b] for b < n and -1 for the padding rows
__global__ void encode_bits(const unsigned long long* __restrict__ ids, int n, int rows, int N, int Kin, bf16* __restrict__ X,
                            const int32_t* __restrict__ lab_in, int32_t* __restrict__ lab_out) {
  hp::pdl_wait();
  hp::pdl_trigger();
  const int b = blockIdx.x * blockDim.y + threadIdx.y;
  if (b >= rows) return;
  if (lab_out && threadIdx.x == 0) lab_out[b] = b < n ? lab_in[b] : -1;
  const unsigned long long g = b < n ? ids[b] : 0ull;
  for (int i = threadIdx.x; i < Kin; i += blockDim.x)
    X[(size_t)b * Kin + i] = __float2bfloat16((b < n && i < N && ((g >> i) & 1ull)) ? 1.f : 0.f);
}

// One block per row: loss += logsumexp(z) - z[label]; dz = (softmax(z) - onehot) * scale (bf16,
// zero in padding columns); rows with label < 0 get dz = 0 and no loss.
// Per labelled row: dZ = (softmax(z) - onehot(label)) * scale (bf16, zero past S and for
// label -1) and the row's loss log(sum exp z) - z[label] added to *loss.  One block per row: an
// online max / sum of exponentials over float4 loads, then one pass writing four bf16 at a time.
__global__ void softmax_xent(const float* __restrict__ Z, int ldz, int S, const int32_t* __restrict__ labels,
                             bf16* __restrict__ dZ, int lddz, int Spad, float scale, float* __restrict__ loss) {
  const int row = blockIdx.x;
  const float* z = Z + (size_t)row * ldz;
  bf16* d = dZ + (size_t)row * lddz;
  const int lab = labels[row];
  __shared__ float red_m[32], red_s[32];
  float m = -INFINITY, sum = 0.f;
  auto add = [&](float v) {  // online update of (max, sum of exp(. - max))
    if (v > m) {
      sum = sum * __expf(m - v) + 1.f;
      m = v;
    } else {
      sum += __expf(v - m);
    }
  };
  const int S4 = S & ~3;
  for (int c = 4 * threadIdx.x; c < S4; c += 4 * blockDim.x) {
    const float4 q = *reinterpret_cast<const float4*>(z + c);
    add(q.x);
    add(q.y);
    add(q.z);
    add(q.w);
  }
  for (int c = S4 + threadIdx.x; c < S; c += blockDim.x) add(z[c]);
  // combine (m, sum) pairs: warp, then block
  for (int o = 16; o; o >>= 1) {
    const float om = __shfl_xor_sync(0xFFFFFFFFu, m, o), os = __shfl_xor_sync(0xFFFFFFFFu, sum, o);
    const float nm = fmaxf(m, om);
    sum = (m == -INFINITY ? 0.f : sum * __expf(m - nm)) + (om == -INFINITY ? 0.f : os * __expf(om - nm));
    m = nm;
  }
  if ((threadIdx.x & 31) == 0) {
    red_m[threadIdx.x >> 5] = m;
    red_s[threadIdx.x >> 5] = sum;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool have = threadIdx.x < (blockDim.x >> 5);
    m = have ? red_m[threadIdx.x] : -INFINITY;
    sum = have ? red_s[threadIdx.x] : 0.f;
    for (int o = 16; o; o >>= 1) {
      const float om = __shfl_xor_sync(0xFFFFFFFFu, m, o), os = __shfl_xor_sync(0xFFFFFFFFu, sum, o);
      const float nm = fmaxf(m, om);
      sum = (m == -INFINITY ? 0.f : sum * __expf(m - nm)) + (om == -INFINITY ? 0.f : os * __expf(om - nm));
      m = nm;
    }
    if (threadIdx.x == 0) {
      red_m[0] = m;
      red_s[0] = sum;
    }
  }
  __syncthreads();
  m = red_m[0];
  sum = red_s[0];
  const float inv = 1.f / sum;
  for (int c = 4 * threadIdx.x; c < Spad; c += 4 * blockDim.x) {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (lab >= 0) {
#pragma unroll
      for (int j = 0; j < 4; j++)
        if (c + j < S) v[j] = (__expf(z[c + j] - m) * inv - (c + j == lab ? 1.f : 0.f)) * scale;
    }
    const __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]), hi = __floats2bfloat162_rn(v[2], v[3]);
    uint2 w;
    w.x = *reinterpret_cast<const uint32_t*>(&lo);
    w.y = *reinterpret_cast<const uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(d + c) = w;
  }
  if (threadIdx.x == 0 && lab >= 0) atomicAdd(loss, logf(sum) + m - z[lab]);
}

// Column sums in two deterministic stages: part[chunk, c] = sum of the chunk's rows (32 rows per
// chunk, two columns per thread from bf16 pairs), then out[c] = sum of part[., c] in chunk order.
constexpr int kColChunk = 32;
__global__ void colsum_partial(const bf16* __restrict__ in, int ld, int rows, int cols, float* __restrict__ part) {
  hp::pdl_wait();
  hp::pdl_trigger();
  const int c = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (c >= cols) return;
  const int r0 = blockIdx.y * kColChunk, r1 = min(rows, r0 + kColChunk);
  float s0 = 0.f, s1 = 0.f;
  if (c + 1 < cols) {
    for (int r = r0; r < r1; r++) {
      const __nv_bfloat162 q = *reinterpret_cast<const __nv_bfloat162*>(in + (size_t)r * ld + c);
      s0 += __low2float(q);
      s1 += __high2float(q);
    }
  } else {
    for (int r = r0; r < r1; r++) s0 += __bfloat162float(in[(size_t)r * ld + c]);
  }
  part[(size_t)blockIdx.y * cols + c] = s0;
  if (c + 1 < cols) part[(size_t)blockIdx.y * cols + c + 1] = s1;
}

// 32 columns per block (lane = column): warp w sums the chunks w, w + 8, ... in order, then the
// eight warp sums are added in warp order
__global__ void colsum_final(const float* __restrict__ part, int chunks, int cols, float* __restrict__ out) {
  hp::pdl_wait();
  hp::pdl_trigger();
  __shared__ float ws[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (c < cols)
    for (int k = w; k < chunks; k += 8) s += part[(size_t)k * cols + c];
  ws[w][lane] = s;
  __syncthreads();
  if (w == 0 && c < cols) {
    float t = 0.f;
#pragma unroll
    for (int i = 0; i < 8; i++) t += ws[i][lane];
    out[c] = t;
  }
}

// out = the sum of the split-K partial products (fp32), slices added in order; four elements per
// thread and step (n and stride multiples of 4, 16-byte aligned buffers)
__global__ void splitk_sum(const float* __restrict__ part, int splits, size_t stride, float* __restrict__ out, size_t n) {
  hp::pdl_wait();
  hp::pdl_trigger();
  for (size_t i = 4 * (blockIdx.x * (size_t)blockDim.x + threadIdx.x); i < n; i += 4 * (size_t)gridDim.x * blockDim.x) {
    float4 v = __ldcs(reinterpret_cast<const float4*>(part + i));
    for (int k = 1; k < splits; k++) {
      const float4 t = __ldcs(reinterpret_cast<const float4*>(part + k * stride + i));
      v.x += t.x;
      v.y += t.y;
      v.z += t.z;
      v.w += t.w;
    }
    *reinterpret_cast<float4*>(out + i) = v;
  }
}

// dA = (sum of the split-K partial products) * (H > 0), bf16 out; four elements per thread and
// step as above
__global__ void splitk_relu_backward(const float* __restrict__ part, int splits, size_t stride, const bf16* __restrict__ H,
                                     bf16* __restrict__ dA, size_t n) {
  hp::pdl_wait();
  hp::pdl_trigger();
  for (size_t i = 4 * (blockIdx.x * (size_t)blockDim.x + threadIdx.x); i < n; i += 4 * (size_t)gridDim.x * blockDim.x) {
    float4 v = __ldcs(reinterpret_cast<const float4*>(part + i));
    for (int k = 1; k < splits; k++) {
      const float4 t = __ldcs(reinterpret_cast<const float4*>(part + k * stride + i));
      v.x += t.x;
      v.y += t.y;
      v.z += t.z;
      v.w += t.w;
    }
    const uint2 h = *reinterpret_cast<const uint2*>(H + i);
    const float hx = __uint_as_float(h.x << 16), hy = __uint_as_float(h.x & 0xFFFF0000u);
    const float hz = __uint_as_float(h.y << 16), hw = __uint_as_float(h.y & 0xFFFF0000u);
    const __nv_bfloat162 lo = __floats2bfloat162_rn(hx > 0.f ? v.x : 0.f, hy > 0.f ? v.y : 0.f);
    const __nv_bfloat162 hi = __floats2bfloat162_rn(hz > 0.f ? v.z : 0.f, hw > 0.f ? v.w : 0.f);
    *reinterpret_cast<uint2*>(dA + i) =
        make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
  }
}

// out[pos, :] = in[perm[pos], :] (rows of H bf16, H a multiple of 8) and bout[pos] = bias[perm[pos]]
__global__ void gather_rows(const bf16* __restrict__ in, const float* __restrict__ bias, const int32_t* __restrict__ perm,
                            int S, int H, bf16* __restrict__ out, float* __restrict__ bout) {
  const size_t chunks = (size_t)H / 8, n = (size_t)S * chunks;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t pos = i / chunks, c = i % chunks;
    const int src = perm[pos];
    reinterpret_cast<uint4*>(out + pos * H)[c] = reinterpret_cast<const uint4*>(in + (size_t)src * H)[c];
    if (c == 0) bout[pos] = bias[src];
  }
}

// dA = dH * (H > 0), fp32 in, bf16 out
__global__ void relu_backward(const float* __restrict__ dH, const bf16* __restrict__ H, bf16* __restrict__ dA, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dA[i] = __float2bfloat16(__bfloat162float(H[i]) > 0.f ? dH[i] : 0.f);
}

// The parameter tensors one Adam launch updates: tensor t holds the elements [end[t-1], end[t])
// of one flat index space (end[-1] = 0)
struct AdamSet {
  float* w[6];
  const float* g[6];
  float* m[6];
  float* v[6];
  bf16* wb[6];  // bf16 copy of w, or null
  size_t end[6];
  int count;
};

__global__ void adam_update(AdamSet s, float lr, float b1, float b2, float eps, float c1, float c2) {
  hp::pdl_wait();
  hp::pdl_trigger();
  const size_t n = s.end[s.count - 1];
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    int t = 0;
    while (k >= s.end[t]) t++;
    const size_t i = k - (t ? s.end[t - 1] : 0);
    float *w = s.w[t], *m = s.m[t], *v = s.v[t];
    const float gi = s.g[t][i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    w[i] = wi;
    if (s.wb[t]) s.wb[t][i] = __float2bfloat16(wi);
  }
}

constexpr int kTopKMax = 16;

// Per row, the k <= KT largest of z[0..S) (ties toward the lower index); one warp per row.  Each
// lane keeps a sorted list of its KT best over a strided, coalesced sweep; then k rounds select
// the largest list head across the warp with shuffles.
template <int KT>
__global__ void topk_warp(const float* __restrict__ Z, int ldz, int S, int k, int rows, int32_t* __restrict__ out) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const float* z = Z + (size_t)row * ldz;
  float bv[KT];
  int bi[KT];
#pragma unroll
  for (int j = 0; j < KT; j++) {
    bv[j] = -INFINITY;
    bi[j] = 0x7FFFFFFF;
  }
  for (int c = lane; c < S; c += 32) {
    const float v = __ldcs(z + c);
    if (v > bv[KT - 1]) {  // equal values arrive in increasing index per lane: the later one never enters
      // insertion into the sorted list (unrolled, branch-free moves)
      float cv = v;
      int ci = c;
#pragma unroll
      for (int j = 0; j < KT; j++) {
        const bool take = cv > bv[j] || (cv == bv[j] && ci < bi[j]);
        const float tv = bv[j];
        const int ti = bi[j];
        bv[j] = take ? cv : bv[j];
        bi[j] = take ? ci : bi[j];
        cv = take ? tv : cv;
        ci = take ? ti : ci;
      }
    }
  }
  for (int r = 0; r < k; r++) {
    float v = bv[0];
    int i = bi[0];
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      const float ov = __shfl_xor_sync(0xFFFFFFFFu, v, off);
      const int oi = __shfl_xor_sync(0xFFFFFFFFu, i, off);
      if (ov > v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
      }
    }
    if (lane == 0) out[(size_t)row * k + r] = i < S ? i : -1;
    if (bi[0] == i) {  // the winning lane pops its head
#pragma unroll
      for (int j = 0; j < KT - 1; j++) {
        bv[j] = bv[j + 1];
        bi[j] = bi[j + 1];
      }
      bv[KT - 1] = -INFINITY;
      bi[KT - 1] = 0x7FFFFFFF;
    }
  }
}

void launch_topk(const float* Z, int ldz, int S, int k, int rows, int32_t* out, cudaStream_t st) {
  const dim3 block(256);
  const dim3 grid((rows + 7) / 8);
  if (k <= 4) topk_warp<4><<<grid, block, 0, st>>>(Z, ldz, S, k, rows, out);
  else if (k <= 8) topk_warp<8><<<grid, block, 0, st>>>(Z, ldz, S, k, rows, out);
  else topk_warp<16><<<grid, block, 0, st>>>(Z, ldz, S, k, rows, out);
}

// cand[r, 2j + q] = q-th conformation of class top[r, j] (or -1)
__global__ void classes_to_conformations(const int32_t* __restrict__ top, long long n, int k,
                                         const int32_t* __restrict__ first_conf, const int32_t* __restrict__ nconf,
                                         int32_t* __restrict__ cand) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n * k) return;
  const int c = top[i];
  const int f = c >= 0 ? first_conf[c] : -1;
  const int m = c >= 0 ? nconf[c] : 0;
  cand[2 * i] = m > 0 ? f : -1;
  cand[2 * i + 1] = m > 1 ? f + 1 : -1;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

// ------------------------------------------------------------------ model

struct hp_mlp {
  int N, H1, H2, S, Kin, Spad, max_batch;
  int device = -1;
  // parameters: fp32 master copies, bf16 working copies, Adam moments, gradients
  float *w[6] = {nullptr}, *g[6] = {nullptr}, *m[6] = {nullptr}, *v[6] = {nullptr};
  size_t n[6] = {0};
  bf16 *w1b = nullptr, *w2b = nullptr, *w3b = nullptr, *w2t = nullptr, *w3t = nullptr;
  // activations / workspaces for max_batch rows (Bp = max_batch rounded to 32)
  bf16 *X = nullptr, *XT = nullptr, *Hb1 = nullptr, *Hb2 = nullptr, *H1T = nullptr, *H2T = nullptr;
  float *Z = nullptr, *dHf = nullptr, *loss = nullptr;
  bf16 *dZ = nullptr, *dZT = nullptr, *dA2 = nullptr, *dA2T = nullptr, *dA1 = nullptr, *dA1T = nullptr;
  int32_t* labels = nullptr;
  unsigned* tc_err = nullptr;  // set by a tcgen05 GEMM whose bounded mbarrier wait gave up
  // fused top-k: per row and 256-class tile range up to 32 candidates (2 lists of up to 16)
  float* cand_v = nullptr;
  int32_t* cand_i = nullptr;
  // column-sum partials (max_batch / 32 + 1 chunks x the widest layer: 256-row chunks of the
  // hidden layers, 32-row blocks of the output layer's gradient) and split-K partial products of
  // the output layer's input gradient (kSplitK x max_batch x H2)
  float* colws = nullptr;
  float* splitws = nullptr;
  // training with the softmax in the output layer's epilogue: per-list row statistics, the
  // label logit, and each row's max and 1 / sum
  float *stats = nullptr, *zlab = nullptr, *row_m = nullptr, *row_inv = nullptr;
  // the proposal's output layer in a scattered class order: neighbouring classes in canonical
  // order are similar folds with similar logits, which would make the fused top-k's running
  // threshold climb slowly along a row; perm[pos] = class at position pos
  int32_t* perm = nullptr;
  bf16* w3p = nullptr;
  float* b3p = nullptr;
  bool w3p_stale = false;  // an optimizer step changed W3 since w3p / b3p were gathered
  int steps = 0;
};

namespace {

// every GEMM runs on the tcgen05 kernel unless HP_MLP_LEGACY_MMA=1 selects the mma.sync kernels
bool tc_enabled() {
  static const bool on = [] {
    const char* e = getenv("HP_MLP_LEGACY_MMA");
    return !(e && e[0] == '1');
  }();
  return on;
}

int gemm(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, const float* bias, int relu, float* Cf,
         int ldcf, bf16* Cb, int ldcb, cudaStream_t st, unsigned* err) {
  if (K % BK != 0 || lda % 8 != 0 || ldb % 8 != 0) return hp::fail(HP_EINVAL, "gemm: K must be a multiple of 32");
  Gemm g{A, B, lda, ldb, M, N, K, bias, relu, Cf, ldcf, Cb, ldcb};
  if (tc_enabled()) {
    hp::TcEpilogue ep;
    ep.bias = bias;
    ep.relu = relu;
    ep.Cf = Cf;
    ep.ldcf = ldcf;
    ep.Cb = Cb;
    ep.ldcb = ldcb;
    return hp::tc_gemm(A, lda, B, ldb, M, N, K, ep, err, st);
  }
  using Big = BigGemm<128, 256, 3>;
  if (K % Big::BK == 0 && (long long)M * N >= (1ll << 22) && K >= 128) {
    cudaFuncSetAttribute(gemm_tn_big<128, 256, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Big::kSmemBytes);
    dim3 grid((N + Big::BN - 1) / Big::BN, (M + Big::BM - 1) / Big::BM);
    gemm_tn_big<128, 256, 3><<<grid, 256, Big::kSmemBytes, st>>>(g);
    return HP_OK;
  }
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  gemm_tn<<<grid, 256, 0, st>>>(g);
  return HP_OK;
}

void transpose(const bf16* in, int ldin, int rows, int cols, bf16* out, int ldout, int out_cols, cudaStream_t st) {
  dim3 grid((cols + 63) / 64, (std::max(rows, out_cols) + 63) / 64);
  transpose_bf16<<<grid, dim3(32, 8), 0, st>>>(in, ldin, rows, cols, out, ldout, out_cols);
}

int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

int sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

constexpr int kSplitK = 8;

// Slices of a split-K GEMM with `tiles` output tiles and nk K chunks: among 1..kmax, the fewest
// that minimise the busiest CTA's chunk count ceil(tiles k / SMs) ceil(nk / k) (one CTA per SM).
int pick_ksplit(int tiles, int nk, int kmax) {
  const int g = sms();
  int best = 1;
  long long best_cost = LLONG_MAX;
  for (int k = 1; k <= std::min(kmax, nk); k++) {
    const long long cost = (long long)((tiles * k + g - 1) / g) * ((nk + k - 1) / k);
    if (cost < best_cost) {
      best_cost = cost;
      best = k;
    }
  }
  return best;
}

// tcgen05 path: a weight gradient out [M x N] = dA^T H over the batch (K rows), with dA stored
// [K][M] (row stride lda) and H stored [K][N] (row stride ldb), both read MN-major.  Few output
// tiles, so K is split over about one CTA per SM and the slices are summed into out.
int weight_grad(hp_mlp* m, const bf16* dA, int lda, const bf16* H, int ldb, int M, int N, int K, float* out,
                cudaStream_t st) {
  const int tiles = ((M + hp::kTcTileM - 1) / hp::kTcTileM) * ((N + hp::kTcTileN - 1) / hp::kTcTileN);
  const int nk = (K + 63) / 64;
  const size_t cap = (size_t)kSplitK * m->max_batch * m->H2;  // splitws floats
  int ks = std::max(1, std::min(nk, sms() / std::max(tiles, 1)));
  while (ks > 1 && (size_t)ks * M * N > cap) ks--;
  hp::TcEpilogue ep;
  ep.a_mn = ep.b_mn = true;
  ep.ldcf = N;
  if (ks == 1) {
    ep.Cf = out;
    return hp::tc_gemm(dA, lda, H, ldb, M, N, K, ep, m->tc_err, st);
  }
  ep.Cf = m->splitws;
  ep.ksplit = ks;
  ep.split_stride = (size_t)M * N;
  const int rc = hp::tc_gemm(dA, lda, H, ldb, M, N, K, ep, m->tc_err, st);
  if (rc == HP_OK)
    hp::launch_pdl(splitk_sum, dim3(grid_for((size_t)M * N / 4)), dim3(256), 0, st, m->splitws, ks, ep.split_stride, out,
                   (size_t)M * N);
  return rc;
}

void colsum(const bf16* in, int ld, int rows, int cols, float* out, float* ws, cudaStream_t st) {
  const int chunks = (rows + kColChunk - 1) / kColChunk;
  hp::launch_pdl(colsum_partial, dim3((cols + 255) / 256, chunks), dim3(128), 0, st, in, ld, rows, cols, ws);
  hp::launch_pdl(colsum_final, dim3((cols + 31) / 32), dim3(256), 0, st, (const float*)ws, chunks, cols, out);
}

// Hidden layers for rows [0, rows) whose ids are in `ids` (n valid) -> m->Hb2; with `labels` (n
// entries) set, they are staged into m->labels (-1 in the padding rows)
int forward_hidden(hp_mlp* m, const unsigned long long* ids, int n, int rows, cudaStream_t st,
                   const int32_t* labels = nullptr) {
  hp::launch_pdl(encode_bits, dim3((rows + 7) / 8), dim3(32, 8), 0, st, ids, n, rows, m->N, m->Kin, m->X, labels,
                 labels ? m->labels : nullptr);
  int rc = gemm(m->X, m->Kin, m->w1b, m->Kin, rows, m->H1, m->Kin, m->w[1], 1, nullptr, 0, m->Hb1, m->H1, st, m->tc_err);
  if (rc == HP_OK)
    rc = gemm(m->Hb1, m->H1, m->w2b, m->H1, rows, m->H2, m->H1, m->w[3], 1, nullptr, 0, m->Hb2, m->H2, st, m->tc_err);
  return rc;
}

// Forward pass: logits -> m->Z (labels staged as in forward_hidden)
int forward(hp_mlp* m, const unsigned long long* ids, int n, int rows, cudaStream_t st, const int32_t* labels = nullptr) {
  int rc = forward_hidden(m, ids, n, rows, st, labels);
  if (rc == HP_OK)
    rc = gemm(m->Hb2, m->H2, m->w3b, m->H2, rows, m->S, m->H2, m->w[5], 0, m->Z, m->Spad, nullptr, 0, st, m->tc_err);
  return rc;
}

// Adam hyper-parameters of one optimizer step (c1, c2: the bias corrections of this step)
struct AdamStep {
  float lr, b1, b2, eps, c1, c2;
};

// mma.sync path (HP_MLP_LEGACY_MMA=1): gradients of the mean cross-entropy over the n valid rows
// into m->g[*] and the loss sum into m->loss, from the logits in m->Z, with transposed copies of
// the operands of the weight gradients
int backward_legacy(hp_mlp* m, int n, int rows, cudaStream_t st) {
  int rc = HP_OK;
  const int S = m->S, H1 = m->H1, H2 = m->H2, Kin = m->Kin, Spad = m->Spad;
  cudaMemsetAsync(m->loss, 0, sizeof(float), st);
  softmax_xent<<<rows, 256, 0, st>>>(m->Z, Spad, S, m->labels, m->dZ, Spad, Spad, 1.f / (float)std::max(n, 1), m->loss);
  // layer 3
  colsum(m->dZ, Spad, rows, S, m->g[5], m->colws, st);
  transpose(m->dZ, Spad, rows, Spad, m->dZT, rows, rows, st);
  transpose(m->Hb2, H2, rows, H2, m->H2T, rows, rows, st);
  if (rc == HP_OK) rc = gemm(m->dZT, rows, m->H2T, rows, S, H2, rows, nullptr, 0, m->g[4], H2, nullptr, 0, st, m->tc_err);
  if (rc == HP_OK) rc = gemm(m->dZ, Spad, m->w3t, Spad, rows, H2, Spad, nullptr, 0, m->dHf, H2, nullptr, 0, st, m->tc_err);
  relu_backward<<<grid_for((size_t)rows * H2), 256, 0, st>>>(m->dHf, m->Hb2, m->dA2, (size_t)rows * H2);
  // layer 2
  colsum(m->dA2, H2, rows, H2, m->g[3], m->colws, st);
  transpose(m->dA2, H2, rows, H2, m->dA2T, rows, rows, st);
  transpose(m->Hb1, H1, rows, H1, m->H1T, rows, rows, st);
  if (rc == HP_OK) rc = gemm(m->dA2T, rows, m->H1T, rows, H2, H1, rows, nullptr, 0, m->g[2], H1, nullptr, 0, st, m->tc_err);
  if (rc == HP_OK) rc = gemm(m->dA2, H2, m->w2t, H2, rows, H1, H2, nullptr, 0, m->dHf, H1, nullptr, 0, st, m->tc_err);
  relu_backward<<<grid_for((size_t)rows * H1), 256, 0, st>>>(m->dHf, m->Hb1, m->dA1, (size_t)rows * H1);
  // layer 1
  colsum(m->dA1, H1, rows, H1, m->g[1], m->colws, st);
  transpose(m->dA1, H1, rows, H1, m->dA1T, rows, rows, st);
  transpose(m->X, Kin, rows, Kin, m->XT, rows, rows, st);
  if (rc == HP_OK) rc = gemm(m->dA1T, rows, m->XT, rows, H1, Kin, rows, nullptr, 0, m->g[0], Kin, nullptr, 0, st, m->tc_err);
  return rc;
}

// tcgen05 path, after the output layer's gradient epilogue has written dZ (and the 32-row column
// sums of dZ into colws): the weight gradients read their operands MN-major (no transposed
// copies), the input gradients read the weights MN-major.  With adam, W3 gets no gradient
// buffer: the GEMM that forms its gradient applies the Adam step and writes W3's bf16 copy, after
// the layer's input gradient has been formed from the old W3.
int backward_tc(hp_mlp* m, int rows, cudaStream_t st, const AdamStep* adam) {
  int rc = HP_OK;
  const int S = m->S, H1 = m->H1, H2 = m->H2, Kin = m->Kin, Spad = m->Spad;
  // layer 3: b3, then dH2 = dZ W3 (rows x H2 with an S-long contraction: too few tiles for the
  // GPU, so split K), then W3's gradient dZ^T H2 (stored or applied)
  hp::launch_pdl(colsum_final, dim3((S + 31) / 32), dim3(256), 0, st, (const float*)m->colws, rows / 32, S, m->g[5]);
  {
    hp::TcEpilogue ep;
    ep.b_mn = true;
    ep.Cf = m->splitws;
    ep.ldcf = H2;
    ep.ksplit = pick_ksplit(((rows + hp::kTcTileM - 1) / hp::kTcTileM) * ((H2 + hp::kTcTileN - 1) / hp::kTcTileN),
                            (S + 63) / 64, kSplitK);
    ep.split_stride = (size_t)rows * H2;
    rc = hp::tc_gemm(m->dZ, Spad, m->w3b, H2, rows, H2, S, ep, m->tc_err, st);
    hp::launch_pdl(splitk_relu_backward, dim3(grid_for((size_t)rows * H2 / 4)), dim3(256), 0, st, (const float*)m->splitws,
                   ep.ksplit, ep.split_stride, (const bf16*)m->Hb2, m->dA2, (size_t)rows * H2);
  }
  {
    hp::TcEpilogue ep;
    ep.a_mn = ep.b_mn = true;
    ep.ldcf = H2;
    if (adam) {
      ep.adam_w = m->w[4];
      ep.adam_m = m->m[4];
      ep.adam_v = m->v[4];
      ep.lr = adam->lr;
      ep.b1 = adam->b1;
      ep.b2 = adam->b2;
      ep.eps = adam->eps;
      ep.c1 = adam->c1;
      ep.c2 = adam->c2;
      ep.Cb = m->w3b;
      ep.ldcb = H2;
    } else {
      ep.Cf = m->g[4];
    }
    if (rc == HP_OK) rc = hp::tc_gemm(m->dZ, Spad, m->Hb2, H2, S, H2, rows, ep, m->tc_err, st);
  }
  // layer 2
  colsum(m->dA2, H2, rows, H2, m->g[3], m->colws, st);
  if (rc == HP_OK) rc = weight_grad(m, m->dA2, H2, m->Hb1, H1, H2, H1, rows, m->g[2], st);
  {
    // dA1 = (dA2 W2) * (H1 > 0), the ReLU's backward step in the GEMM's epilogue
    hp::TcEpilogue ep;
    ep.b_mn = true;
    ep.Cb = m->dA1;
    ep.ldcb = H1;
    ep.relu_mask = m->Hb1;
    ep.ldmask = H1;
    if (rc == HP_OK) rc = hp::tc_gemm(m->dA2, H2, m->w2b, H1, rows, H1, H2, ep, m->tc_err, st);
  }
  // layer 1
  colsum(m->dA1, H1, rows, H1, m->g[1], m->colws, st);
  if (rc == HP_OK) rc = weight_grad(m, m->dA1, H1, m->X, Kin, H1, Kin, rows, m->g[0], st);
  return rc;
}

// Loss and gradients of one batch.  On the tcgen05 path the softmax runs in the output layer's
// epilogue: a first pass of the layer's GEMM keeps per-row maxima and sums of exponentials, a
// second pass recomputes the logits and writes their gradient (and its 32-row column sums), so
// the fp32 logits never reach memory.
int loss_and_gradients(hp_mlp* m, const unsigned long long* ids, const int32_t* labels, int n, int rows, cudaStream_t st,
                       const AdamStep* adam = nullptr) {
  if (!tc_enabled()) {
    int rc = forward(m, ids, n, rows, st, labels);
    if (rc == HP_OK) rc = backward_legacy(m, n, rows, st);
    return rc;
  }
  int rc = forward_hidden(m, ids, n, rows, st, labels);
  hp::TcEpilogue ea;
  ea.kt = -1;
  ea.bias = m->w[5];
  ea.labels = m->labels;
  ea.stats = m->stats;
  ea.zlab = m->zlab;
  if (rc == HP_OK) rc = hp::tc_gemm(m->Hb2, m->H2, m->w3b, m->H2, rows, m->S, m->H2, ea, m->tc_err, st);
  if (rc != HP_OK) return rc;
  cudaMemsetAsync(m->loss, 0, sizeof(float), st);
  hp::tc_softmax_finish(m->stats, hp::tc_stats_lists(rows, m->S), rows, m->labels, m->zlab, m->row_m, m->row_inv, m->loss,
                        st);
  hp::TcEpilogue eb;
  eb.kt = -2;
  eb.bias = m->w[5];
  eb.labels = m->labels;
  eb.row_m = m->row_m;
  eb.row_inv = m->row_inv;
  eb.zlab = m->zlab;
  eb.scale = 1.f / (float)std::max(n, 1);
  eb.dz = m->dZ;
  eb.ldz = m->Spad;
  eb.colpart = m->colws;
  rc = hp::tc_gemm(m->Hb2, m->H2, m->w3b, m->H2, rows, m->S, m->H2, eb, m->tc_err, st);
  if (rc == HP_OK) rc = backward_tc(m, rows, st, adam);
  return rc;
}

// the output layer's weights and biases in the top-k GEMM's scattered class order
void gather_w3p(hp_mlp* m, cudaStream_t st) {
  gather_rows<<<grid_for((size_t)m->S * (m->H2 / 8)), 256, 0, st>>>(m->w3b, m->w[5], m->perm, m->S, m->H2, m->w3p, m->b3p);
  m->w3p_stale = false;
}

// refresh the bf16 copies used by the GEMMs (cast: the plain bf16 copies, which the optimizer
// step writes itself; the mma.sync path also needs the weights' transposes); the scattered copy
// for the top-k is gathered here when cast is set and otherwise marked stale, for the next top-k
// call
void refresh_copies(hp_mlp* m, cudaStream_t st, bool cast = true) {
  if (cast) {
    cast_bf16<<<grid_for(m->n[0]), 256, 0, st>>>(m->w[0], m->w1b, m->n[0]);
    cast_bf16<<<grid_for(m->n[2]), 256, 0, st>>>(m->w[2], m->w2b, m->n[2]);
    cast_bf16<<<grid_for(m->n[4]), 256, 0, st>>>(m->w[4], m->w3b, m->n[4]);
  }
  if (!tc_enabled()) {
    transpose(m->w2b, m->H1, m->H2, m->H1, m->w2t, m->H2, m->H2, st);
    transpose(m->w3b, m->H2, m->S, m->H2, m->w3t, m->Spad, m->Spad, st);
  }
  if (cast)
    gather_w3p(m, st);
  else
    m->w3p_stale = true;
}

void free_model(hp_mlp* m) {
  if (!m) return;
  for (int i = 0; i < 6; i++) {
    cudaFree(m->w[i]);
    cudaFree(m->g[i]);
    cudaFree(m->m[i]);
    cudaFree(m->v[i]);
  }
  void* ptrs[] = {m->w1b, m->w2b, m->w3b, m->w2t, m->w3t, m->X,  m->XT,  m->Hb1, m->Hb2,  m->H1T,  m->H2T,
                  m->Z,   m->dHf, m->loss, m->dZ,  m->dZT, m->dA2, m->dA2T, m->dA1, m->dA1T, m->labels, m->tc_err, m->cand_v, m->cand_i,
                  m->colws, m->splitws, m->stats, m->zlab, m->row_m, m->row_inv, m->perm, m->w3p, m->b3p};
  for (void* p : ptrs) cudaFree(p);
  delete m;
}

}  // namespace

extern "C" int hp_mlp_create(int32_t N, int32_t H1, int32_t H2, int32_t S, int32_t max_batch, const float* const* h_params,
                             hp_mlp** out) {
  if (!out) return hp::fail(HP_EINVAL, "hp_mlp_create: out is NULL");
  *out = nullptr;
  if (N < 1 || N > 64 || H1 < 32 || H2 < 32 || H1 % 32 || H2 % 32 || S < 1 || max_batch < 1 || !h_params)
    return hp::fail(HP_EINVAL, "hp_mlp_create: bad sizes (hidden widths must be multiples of 32)");
  hp_mlp* m = new (std::nothrow) hp_mlp();
  if (!m) return hp::fail(HP_ENOMEM, "hp_mlp_create: out of host memory");
  m->N = N;
  m->H1 = H1;
  m->H2 = H2;
  m->S = S;
  m->Kin = round_up(N, 32);
  m->Spad = round_up(S, 32);
  m->max_batch = round_up(max_batch, 32);
  cudaGetDevice(&m->device);
  const size_t B = m->max_batch;
  // W1 [H1, Kin] (columns >= N zero), b1 [H1], W2 [H2, H1], b2 [H2], W3 [S, H2], b3 [S]
  m->n[0] = (size_t)H1 * m->Kin;
  m->n[1] = H1;
  m->n[2] = (size_t)H2 * H1;
  m->n[3] = H2;
  m->n[4] = (size_t)S * H2;
  m->n[5] = S;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 6 && e == cudaSuccess; i++) {
    e = cudaMalloc(&m->w[i], m->n[i] * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->g[i], m->n[i] * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->m[i], m->n[i] * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->v[i], m->n[i] * 4);
    if (e == cudaSuccess) e = cudaMemset(m->m[i], 0, m->n[i] * 4);
    if (e == cudaSuccess) e = cudaMemset(m->v[i], 0, m->n[i] * 4);
  }
  auto al = [&](auto** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
  };
  al(&m->w1b, m->n[0] * 2);
  al(&m->w2b, m->n[2] * 2);
  al(&m->w3b, m->n[4] * 2);
  al(&m->X, B * m->Kin * 2);
  al(&m->Hb1, B * H1 * 2);
  al(&m->Hb2, B * H2 * 2);
  al(&m->Z, B * m->Spad * 4);
  al(&m->dHf, B * std::max(H1, H2) * 4);
  al(&m->loss, 4);
  al(&m->dZ, B * m->Spad * 2);
  al(&m->dA2, B * H2 * 2);
  al(&m->dA1, B * H1 * 2);
  if (!tc_enabled()) {
    // the mma.sync path's transposed copies (the tcgen05 GEMMs read these operands MN-major)
    al(&m->w2t, (size_t)H1 * H2 * 2);
    al(&m->w3t, (size_t)H2 * m->Spad * 2);
    al(&m->XT, (size_t)m->Kin * B * 2);
    al(&m->H1T, (size_t)H1 * B * 2);
    al(&m->H2T, (size_t)H2 * B * 2);
    al(&m->dZT, (size_t)m->Spad * B * 2);
    al(&m->dA2T, (size_t)H2 * B * 2);
    al(&m->dA1T, (size_t)H1 * B * 2);
  }
  al(&m->labels, B * 4);
  al(&m->tc_err, sizeof(unsigned));
  const size_t ncand = (size_t)max_batch * ((S + hp::kTcTileN - 1) / hp::kTcTileN) * hp::kTcTopkSlotsPerTile;
  al(&m->cand_v, ncand * 4);
  al(&m->cand_i, ncand * 4);
  al(&m->colws, (size_t)(B / 32 + 1) * std::max(m->Spad, std::max(H1, H2)) * 4);
  al(&m->splitws, (size_t)kSplitK * B * H2 * 4);
  al(&m->stats, (size_t)((S + hp::kTcTileN - 1) / hp::kTcTileN) * hp::kTcStatsListsPerTile * B * 2 * 4);
  al(&m->zlab, B * 4);
  al(&m->row_m, B * 4);
  al(&m->row_inv, B * 4);
  al(&m->perm, (size_t)S * 4);
  al(&m->w3p, m->n[4] * 2);
  al(&m->b3p, (size_t)S * 4);
  if (e != cudaSuccess) {
    free_model(m);
    return hp::cuda_fail(e, "hp_mlp_create: device allocation");
  }
  // parameters from the host: W1 arrives as [H1, N] and is widened to [H1, Kin]
  std::vector<float> w1((size_t)H1 * m->Kin, 0.f);
  for (int r = 0; r < H1; r++)
    for (int c = 0; c < N; c++) w1[(size_t)r * m->Kin + c] = h_params[0][(size_t)r * N + c];
  e = cudaMemcpy(m->w[0], w1.data(), w1.size() * 4, cudaMemcpyHostToDevice);
  for (int i = 1; i < 6 && e == cudaSuccess; i++) e = cudaMemcpy(m->w[i], h_params[i], m->n[i] * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_model(m);
    return hp::cuda_fail(e, "hp_mlp_create: upload");
  }
  {
    // multiplicative scatter pos -> (pos * a) mod S with a near 0.618 S and coprime to S
    long long a = std::max(1ll, (long long)(0.6180339887 * S));
    while (std::gcd(a, (long long)S) != 1) a++;
    std::vector<int32_t> perm(S);
    for (int pos = 0; pos < S; pos++) perm[pos] = (int32_t)(((long long)pos * a) % S);
    e = cudaMemcpy(m->perm, perm.data(), (size_t)S * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      free_model(m);
      return hp::cuda_fail(e, "hp_mlp_create: upload");
    }
  }
  refresh_copies(m, nullptr);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_model(m);
    return hp::cuda_fail(e, "hp_mlp_create");
  }
  *out = m;
  return HP_OK;
}

extern "C" void hp_mlp_free(hp_mlp* m) { free_model(m); }

namespace {
// read (and clear) the tcgen05 timeout word after the stream has drained
int take_status(hp_mlp* m, cudaStream_t st, const char* what) {
  unsigned flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, m->tc_err, sizeof(flag), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && flag) e = cudaMemsetAsync(m->tc_err, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return hp::cuda_fail(e, what);
  if (flag) return hp::fail(HP_ETIMEOUT, "tcgen05 GEMM: bounded mbarrier wait gave up (results invalid)");
  return HP_OK;
}
}  // namespace

extern "C" int hp_mlp_status(hp_mlp* m, void* stream) {
  if (!m) return hp::fail(HP_EINVAL, "hp_mlp_status: NULL model");
  return take_status(m, (cudaStream_t)stream, "hp_mlp_status");
}

extern "C" int hp_mlp_gradients(hp_mlp* m, const uint64_t* d_ids, const int32_t* d_labels, int32_t n,
                                 float* const* h_grads, float* h_loss, void* stream) {
  if (!m || !d_ids || !d_labels) return hp::fail(HP_EINVAL, "hp_mlp_gradients: NULL argument");
  if (n < 1 || n > m->max_batch) return hp::fail(HP_EINVAL, "hp_mlp_gradients: batch exceeds max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  const int rows = round_up(n, 32);
  int rc = loss_and_gradients(m, reinterpret_cast<const unsigned long long*>(d_ids), d_labels, n, rows, st);
  if (rc != HP_OK) return rc;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_mlp_gradients: launch");
  if (h_grads) {
    std::vector<float> g1(m->n[0]);
    e = cudaMemcpyAsync(g1.data(), m->g[0], m->n[0] * 4, cudaMemcpyDeviceToHost, st);
    for (int i = 1; i < 6 && e == cudaSuccess; i++)
      if (h_grads[i]) e = cudaMemcpyAsync(h_grads[i], m->g[i], m->n[i] * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && h_grads[0])
      for (int r = 0; r < m->H1; r++)
        for (int c = 0; c < m->N; c++) h_grads[0][(size_t)r * m->N + c] = g1[(size_t)r * m->Kin + c];
  }
  if (h_loss && e == cudaSuccess) {
    float l = 0;
    e = cudaMemcpyAsync(&l, m->loss, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    *h_loss = l / (float)n;
  }
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_mlp_gradients");
  if (h_grads || h_loss) return take_status(m, st, "hp_mlp_gradients");
  return HP_OK;
}

extern "C" int hp_mlp_train_step(hp_mlp* m, const uint64_t* d_ids, const int32_t* d_labels, int32_t n, float lr,
                                 float* h_loss, void* stream) {
  if (!m || !d_ids || !d_labels) return hp::fail(HP_EINVAL, "hp_mlp_train_step: NULL argument");
  if (n < 1 || n > m->max_batch) return hp::fail(HP_EINVAL, "hp_mlp_train_step: batch exceeds max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  const int rows = round_up(n, 32);
  const int step = m->steps + 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const AdamStep adam{lr, b1, b2, eps, 1.f / (1.f - powf(b1, (float)step)), 1.f / (1.f - powf(b2, (float)step))};
  // on the tcgen05 path W3's update is fused into the GEMM that forms its gradient
  const bool fused = tc_enabled();
  int rc = loss_and_gradients(m, reinterpret_cast<const unsigned long long*>(d_ids), d_labels, n, rows, st,
                              fused ? &adam : nullptr);
  if (rc != HP_OK) return rc;
  m->steps = step;
  // the weight matrices' bf16 copies are written by the update itself
  bf16* const wb[6] = {m->w1b, nullptr, m->w2b, nullptr, m->w3b, nullptr};
  AdamSet set{};
  size_t total = 0;
  for (int i = 0; i < 6; i++)
    if (!(fused && i == 4)) {
      const int t = set.count++;
      set.w[t] = m->w[i];
      set.g[t] = m->g[i];
      set.m[t] = m->m[i];
      set.v[t] = m->v[i];
      set.wb[t] = wb[i];
      set.end[t] = total += m->n[i];
    }
  hp::launch_pdl(adam_update, dim3(grid_for(total)), dim3(256), 0, st, set, adam.lr, adam.b1, adam.b2, adam.eps, adam.c1,
                 adam.c2);
  refresh_copies(m, st, false);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_mlp_train_step: launch");
  if (h_loss) {
    float l = 0;
    e = cudaMemcpyAsync(&l, m->loss, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return hp::cuda_fail(e, "hp_mlp_train_step");
    *h_loss = l / (float)n;
    return take_status(m, st, "hp_mlp_train_step");
  }
  return HP_OK;
}

extern "C" int hp_mlp_topk(hp_mlp* m, const uint64_t* d_ids, int64_t n, int32_t k, int32_t* d_top, void* stream) {
  if (!m || !d_ids || !d_top) return hp::fail(HP_EINVAL, "hp_mlp_topk: NULL argument");
  if (k < 1 || k > kTopKMax || k > m->S) return hp::fail(HP_EINVAL, "hp_mlp_topk: k must be in [1, 16] and <= S");
  cudaStream_t st = (cudaStream_t)stream;
  if (tc_enabled() && m->w3p_stale) gather_w3p(m, st);
  for (int64_t off = 0; off < n; off += m->max_batch) {
    const int nb = (int)std::min<int64_t>(m->max_batch, n - off);
    const int rows = round_up(nb, 32);
    const unsigned long long* ids = reinterpret_cast<const unsigned long long*>(d_ids) + off;
    if (tc_enabled()) {
      // output layer with the top-k fused into the GEMM epilogue: logits never reach memory
      int rc = forward_hidden(m, ids, nb, rows, st);
      hp::TcEpilogue ep;
      ep.bias = m->b3p;
      ep.kt = k <= 4 ? 4 : k <= 8 ? 8 : 16;
      ep.cand_v = m->cand_v;
      ep.cand_i = m->cand_i;
      ep.col_id = m->perm;
      if (rc == HP_OK) rc = hp::tc_gemm(m->Hb2, m->H2, m->w3p, m->H2, nb, m->S, m->H2, ep, m->tc_err, st);
      if (rc != HP_OK) return rc;
      hp::tc_topk_merge(m->cand_v, m->cand_i, hp::tc_topk_lists(nb, m->S, ep.kt), nb, ep.kt, k, m->S, d_top + off * k, st);
    } else {
      int rc = forward(m, ids, nb, rows, st);
      if (rc != HP_OK) return rc;
      launch_topk(m->Z, m->Spad, m->S, k, nb, d_top + off * k, st);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_mlp_topk: launch");
  return HP_OK;
}

extern "C" int hp_mlp_logits(hp_mlp* m, const uint64_t* d_ids, int32_t n, float* d_logits, void* stream) {
  if (!m || !d_ids || !d_logits || n < 1 || n > m->max_batch) return hp::fail(HP_EINVAL, "hp_mlp_logits: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = forward(m, reinterpret_cast<const unsigned long long*>(d_ids), n, round_up(n, 32), st);
  if (rc != HP_OK) return rc;
  cudaError_t e = cudaMemcpy2DAsync(d_logits, (size_t)m->S * 4, m->Z, (size_t)m->Spad * 4, (size_t)m->S * 4, n,
                                    cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_mlp_logits");
  return HP_OK;
}

extern "C" int hp_proposal_conformations(const hp_structs* s, const int32_t* d_top, int64_t n, int32_t k, int32_t* d_cand,
                                         void* stream) {
  if (!s || !d_top || !d_cand) return hp::fail(HP_EINVAL, "hp_proposal_conformations: NULL argument");
  if (n < 0 || k < 1) return hp::fail(HP_EINVAL, "hp_proposal_conformations: n must be >= 0 and k >= 1");
  hp::DevTables* dt = nullptr;
  int rc = hp::device_tables(s, &dt);
  if (rc != HP_OK) return rc;
  hp_structs* ms = const_cast<hp_structs*>(s);
  std::lock_guard<std::mutex> lock(ms->mu);
  if (!dt->class_first) {
    std::vector<int32_t> first(s->S, -1), cnt(s->S, 0);
    for (int32_t c = s->S_dir - 1; c >= 0; c--) {
      first[s->conf_class[c]] = c;
      cnt[s->conf_class[c]]++;
    }
    cudaError_t e = cudaMalloc(&dt->class_first, (size_t)s->S * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dt->class_nconf, (size_t)s->S * 4);
    if (e == cudaSuccess) e = cudaMemcpy(dt->class_first, first.data(), (size_t)s->S * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dt->class_nconf, cnt.data(), (size_t)s->S * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      // leave no half-built table behind: the next call rebuilds both
      cudaFree(dt->class_first);
      cudaFree(dt->class_nconf);
      dt->class_first = nullptr;
      dt->class_nconf = nullptr;
      return hp::cuda_fail(e, "hp_proposal_conformations: class tables");
    }
  }
  const long long total = n * (long long)k;
  if (total > 0)
    classes_to_conformations<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        d_top, n, k, dt->class_first, dt->class_nconf, d_cand);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_proposal_conformations: launch");
  return HP_OK;
}
