// Batched persistent launch, CUDA-graph plans and the kernel-shape autotuner.
//
// Several boxes (fold libraries of different shapes and sizes) and sequence
// ranges are planned into one work list and computed by one persistent launch
// of the phenotype kernel; CTAs pull work items from a device counter, the
// boxes with more conformations first.  A plan captures the counter reset and
// that launch into a CUDA graph once, so repeated batches replay it without
// per-launch host work.  The autotuner times every supported kernel shape
// (sequences per thread x conformations per shared-memory tile) on a bounded
// number of work items and keeps the fastest on the library handle.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hp_internal.h"
#include "phenotype.h"

namespace {

const int kShapes[][2] = {{4, 64}, {4, 128}, {5, 64}, {5, 128}, {5, 256}, {6, 64}, {6, 128}, {6, 256}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

int shape_of(const hp_tile_cfg* cfg, const hp_structs* first, int* r, int* t) {
  if (cfg) {
    *r = cfg->reg_bits;
    *t = cfg->tile;
  } else if (first && first->tile_reg_bits) {
    *r = first->tile_reg_bits;
    *t = first->tile_size;
  } else {
    hp::default_tile_cfg(r, t);
  }
  if (!hp::tile_cfg_supported(*r, *t))
    return hp::fail(HP_EINVAL, "tile configuration (reg_bits " + std::to_string(*r) + ", tile " + std::to_string(*t) +
                                   ") is not one of the compiled shapes");
  return HP_OK;
}

}  // namespace

struct hp_batch_plan {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  std::vector<unsigned*> ctrl;  // one control block per captured launch (role class)
  int device = -1;
};

extern "C" int hp_set_tile_cfg(hp_structs* s, const hp_tile_cfg* cfg) {
  if (!s) return hp::fail(HP_EINVAL, "hp_set_tile_cfg: library is NULL");
  if (!cfg) {
    s->tile_reg_bits = 0;
    s->tile_size = 0;
    return HP_OK;
  }
  if (!hp::tile_cfg_supported(cfg->reg_bits, cfg->tile))
    return hp::fail(HP_EINVAL, "hp_set_tile_cfg: not one of the compiled shapes");
  s->tile_reg_bits = cfg->reg_bits;
  s->tile_size = cfg->tile;
  return HP_OK;
}

extern "C" int hp_get_tile_cfg(const hp_structs* s, hp_tile_cfg* cfg) {
  if (!s || !cfg) return hp::fail(HP_EINVAL, "hp_get_tile_cfg: NULL argument");
  int r = s->tile_reg_bits, t = s->tile_size;
  if (!r) hp::default_tile_cfg(&r, &t);
  cfg->reg_bits = r;
  cfg->tile = t;
  return HP_OK;
}

extern "C" int hp_tile_cfg_list(hp_tile_cfg* cfgs, int32_t* n) {
  if (!n) return hp::fail(HP_EINVAL, "hp_tile_cfg_list: n is NULL");
  if (cfgs)
    for (int i = 0; i < kNumShapes && i < *n; i++) {
      cfgs[i].reg_bits = kShapes[i][0];
      cfgs[i].tile = kShapes[i][1];
    }
  *n = kNumShapes;
  return HP_OK;
}

extern "C" int hp_phenotype_map_batch(const hp_structs* const* libs, const uint64_t* begins, const uint64_t* counts,
                                      int32_t n, int32_t* const* d_phen, const hp_tile_cfg* cfg, void* stream) {
  if (!libs || !begins || !counts || !d_phen) return hp::fail(HP_EINVAL, "hp_phenotype_map_batch: NULL argument");
  if (n < 1) return hp::fail(HP_EINVAL, "hp_phenotype_map_batch: empty batch");
  int r = 0, t = 0;
  int rc = shape_of(cfg, libs[0], &r, &t);
  if (rc != HP_OK) return rc;
  // no shape given: the role count follows the blocks (all boxes of the launch share it)
  const bool auto_roles = !cfg && !libs[0]->tile_reg_bits;
  return hp::run_phenotype(libs, begins, counts, n, d_phen, nullptr, r, t, (cudaStream_t)stream, 0, 1, auto_roles);
}

extern "C" int hp_phenotype_map_batch_gap(const hp_structs* const* libs, const uint64_t* begins, const uint64_t* counts,
                                          int32_t n, int32_t gap_threshold, int32_t* const* d_phen, void* stream) {
  if (!libs || !begins || !counts || !d_phen) return hp::fail(HP_EINVAL, "hp_phenotype_map_batch_gap: NULL argument");
  if (n < 1) return hp::fail(HP_EINVAL, "hp_phenotype_map_batch_gap: empty batch");
  if (gap_threshold < 1 || gap_threshold > (1 << 20))
    return hp::fail(HP_EINVAL, "hp_phenotype_map_batch_gap: gap_threshold must be in [1, 2^20]");
  int r = 0, t = 0;
  hp::default_tile_cfg(&r, &t);
  return hp::run_phenotype(libs, begins, counts, n, d_phen, nullptr, r, t, (cudaStream_t)stream, 0, gap_threshold,
                           gap_threshold == 1);
}

extern "C" int hp_autotune(hp_structs* s, hp_tile_cfg* best, float* ms, void* stream) {
  if (!s) return hp::fail(HP_EINVAL, "hp_autotune: library is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  // an aligned block of at most 2^28 ids: every work item covers 2^14 sequences whatever the shape
  const uint64_t begin = 0, count = 1ull << (s->N < 28 ? s->N : 28);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // two waves of work items (every shape covers 2^14 sequences per item); outputs go to scratch
  const unsigned grid = (unsigned)(sms > 0 ? sms : 1);
  hp::PhenParams* prm = new (std::nothrow) hp::PhenParams();
  if (!prm) return hp::fail(HP_ENOMEM, "hp_autotune: out of host memory");
  int32_t* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, sizeof(int32_t) * (size_t)count, st);
  if (e != cudaSuccess) {
    delete prm;
    return hp::cuda_fail(e, "hp_autotune: cudaMallocAsync");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 0;
  int best_i = -1, rc = HP_OK;
  unsigned herr = 0;
  const hp_structs* cs = s;
  for (int i = 0; i < kNumShapes && rc == HP_OK; i++) {
    rc = hp::plan_phenotype(&cs, &begin, &count, 1, &scratch, nullptr, kShapes[i][1], *prm);
    if (rc != HP_OK) break;
    const unsigned long long limit = 2ull * grid;
    if (prm->total_items > limit) prm->total_items = limit;
    float t_ms = -1;
    size_t bytes = 0;
    unsigned ctas = 0;
    void* block = nullptr;
    if (hp::launch_block_bytes(*prm, kShapes[i][0], kShapes[i][1], grid, &bytes, &ctas) != HP_OK) {
      // a shape that does not fit this device is skipped, not fatal
      if (ms) ms[i] = -1;
      continue;
    }
    e = cudaMallocAsync(&block, bytes, st);
    if (e != cudaSuccess) {
      rc = hp::cuda_fail(e, "hp_autotune: cudaMallocAsync(control words and work lists)");
      break;
    }
    hp::bind_launch_block(*prm, block, ctas);
    for (int rep = 0; rep < 2 && rc == HP_OK; rep++) {  // first run warms up
      cudaMemsetAsync(prm->ctrl, 0, hp::kPhenCtrlBytes, st);
      cudaEventRecord(e0, st);
      rc = hp::launch_phenotype(*prm, kShapes[i][0], kShapes[i][1], st, grid);
      cudaEventRecord(e1, st);
      if (rc == HP_OK) {
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_autotune: timing run");
        cudaEventElapsedTime(&t_ms, e0, e1);
      }
    }
    if (rc == HP_OK) {
      unsigned h = 0;
      e = cudaMemcpyAsync(&h, prm->ctrl, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_autotune");
      herr |= h;
    }
    cudaFreeAsync(block, st);
    if (ms) ms[i] = t_ms;
    if (rc == HP_OK && t_ms > 0 && (best_i < 0 || t_ms < best_ms)) {
      best_ms = t_ms;
      best_i = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(scratch, st);
  delete prm;
  if (rc != HP_OK) return rc;
  if (herr) return hp::fail(HP_ETIMEOUT, "hp_autotune: a timing run reported a device-side timeout");
  if (best_i < 0) return hp::fail(HP_EUNSUPPORTED, "hp_autotune: no kernel shape fits this device");
  s->tile_reg_bits = kShapes[best_i][0];
  s->tile_size = kShapes[best_i][1];
  if (best) {
    best->reg_bits = s->tile_reg_bits;
    best->tile = s->tile_size;
  }
  return HP_OK;
}

extern "C" int hp_batch_plan_create(const hp_structs* const* libs, const uint64_t* begins, const uint64_t* counts,
                                    int32_t n, int32_t* const* d_phen, const hp_tile_cfg* cfg, void* stream,
                                    hp_batch_plan** out) {
  if (!out) return hp::fail(HP_EINVAL, "hp_batch_plan_create: out is NULL");
  *out = nullptr;
  if (!libs || !begins || !counts || !d_phen || n < 1) return hp::fail(HP_EINVAL, "hp_batch_plan_create: bad batch");
  int r = 0, t = 0;
  int rc = shape_of(cfg, libs[0], &r, &t);
  if (rc != HP_OK) return rc;
  hp_batch_plan* plan = new (std::nothrow) hp_batch_plan();
  if (!plan) return hp::fail(HP_ENOMEM, "hp_batch_plan_create: out of host memory");
  cudaGetDevice(&plan->device);
  // no shape given: boxes are grouped by role count, one persistent launch per group (all in the graph)
  std::vector<int> cls(n, 14);
  const bool auto_roles = !cfg && !libs[0]->tile_reg_bits;
  if (auto_roles) rc = hp::role_classes(libs, begins, counts, n, d_phen, t, cls);
  // plans (tables are uploaded here, before capture begins) and their device blocks
  std::vector<hp::PhenParams*> prms;
  std::vector<int> shape_r, shape_t;
  for (const int c : {14, 13, 12, 11}) {
    if (rc != HP_OK) break;
    std::vector<const hp_structs*> l;
    std::vector<uint64_t> bg, ct;
    std::vector<int32_t*> o;
    for (int i = 0; i < n; i++)
      if (cls[i] == c) {
        l.push_back(libs[i]);
        bg.push_back(begins[i]);
        ct.push_back(counts[i]);
        o.push_back(d_phen[i]);
      }
    if (l.empty()) continue;
    int r2 = r, t2 = t, roles = 14;
    if (c != 14) hp::small_roles_shape(c, &roles, &r2, &t2);
    hp::PhenParams* prm = new (std::nothrow) hp::PhenParams();
    if (!prm) {
      rc = hp::fail(HP_ENOMEM, "hp_batch_plan_create: out of host memory");
      break;
    }
    prms.push_back(prm);
    shape_r.push_back(r2);
    shape_t.push_back(t2);
    rc = hp::plan_phenotype(l.data(), bg.data(), ct.data(), (int)l.size(), o.data(), nullptr, t2, *prm, c);
    if (rc != HP_OK) break;
    size_t bytes = hp::kPhenCtrlBytes;
    unsigned ctas = 0;
    if (prm->total_items) rc = hp::launch_block_bytes(*prm, r2, t2, 0, &bytes, &ctas);
    if (rc != HP_OK) break;
    unsigned* block = nullptr;
    cudaError_t e = cudaMalloc(&block, bytes);
    if (e != cudaSuccess) {
      rc = hp::cuda_fail(e, "hp_batch_plan_create: cudaMalloc");
      break;
    }
    plan->ctrl.push_back(block);
    if (prm->total_items) hp::bind_launch_block(*prm, block, ctas);
  }
  cudaStream_t cap = nullptr;
  cudaError_t e = cudaSuccess;
  if (rc == HP_OK) {
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_batch_plan_create: cudaStreamCreate");
  }
  if (rc == HP_OK) {
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      int lrc = HP_OK;
      for (size_t q = 0; q < prms.size() && lrc == HP_OK; q++) {
        cudaMemsetAsync(plan->ctrl[q], 0, hp::kPhenCtrlBytes, cap);
        if (prms[q]->total_items) lrc = hp::launch_phenotype(*prms[q], shape_r[q], shape_t[q], cap, 0);
      }
      cudaError_t e2 = cudaStreamEndCapture(cap, &plan->graph);
      if (lrc != HP_OK) rc = lrc;
      else if (e2 != cudaSuccess) rc = hp::cuda_fail(e2, "hp_batch_plan_create: cudaStreamEndCapture");
    } else {
      rc = hp::cuda_fail(e, "hp_batch_plan_create: cudaStreamBeginCapture");
    }
  }
  if (rc == HP_OK) {
    e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
    if (e != cudaSuccess) rc = hp::cuda_fail(e, "hp_batch_plan_create: cudaGraphInstantiate");
  }
  if (cap) cudaStreamDestroy(cap);
  for (hp::PhenParams* prm : prms) delete prm;
  (void)stream;
  if (rc != HP_OK) {
    hp_batch_plan_free(plan);
    return rc;
  }
  *out = plan;
  return HP_OK;
}

extern "C" int hp_batch_plan_launch(hp_batch_plan* plan, void* stream) {
  if (!plan || !plan->exec) return hp::fail(HP_EINVAL, "hp_batch_plan_launch: invalid plan");
  cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_batch_plan_launch: cudaGraphLaunch");
  return HP_OK;
}

extern "C" int hp_batch_plan_status(hp_batch_plan* plan, void* stream) {
  if (!plan || plan->ctrl.empty()) return hp::fail(HP_EINVAL, "hp_batch_plan_status: invalid plan");
  std::vector<unsigned> herr(plan->ctrl.size(), 0u);
  cudaError_t e = cudaSuccess;
  for (size_t q = 0; q < plan->ctrl.size() && e == cudaSuccess; q++)
    e = cudaMemcpyAsync(&herr[q], plan->ctrl[q], sizeof(unsigned), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return hp::cuda_fail(e, "hp_batch_plan_status");
  for (unsigned h : herr)
    if (h) return hp::fail(HP_ETIMEOUT, "hp_batch_plan_status: a bounded device wait timed out");
  return HP_OK;
}

extern "C" void hp_batch_plan_free(hp_batch_plan* plan) {
  if (!plan) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (plan->device >= 0) cudaSetDevice(plan->device);
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  for (unsigned* c : plan->ctrl) cudaFree(c);
  if (cur >= 0 && plan->device >= 0) cudaSetDevice(cur);
  delete plan;
}
