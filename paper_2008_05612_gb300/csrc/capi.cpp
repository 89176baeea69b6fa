// Status handling and per-device tables shared by the C entry points.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <new>
#include <string>

#include "hp_internal.h"

namespace {
thread_local std::string g_last_error = "no error";
std::atomic<long long> g_wait_limit{-1};  // < 0: every kernel uses its own constant
}

namespace hp {

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(int err, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString((cudaError_t)err);
  return err == cudaErrorMemoryAllocation ? HP_ENOMEM : HP_ECUDA;
}

long long wait_limit(long long dflt) {
  const long long v = g_wait_limit.load(std::memory_order_relaxed);
  return v < 0 ? dflt : v;
}

int device_tables(const hp_structs* cs, DevTables** out) {
  hp_structs* s = const_cast<hp_structs*>(cs);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(s->mu);
  for (DevTables* t : s->dev)
    if (t->device == dev) {
      *out = t;
      return HP_OK;
    }
  DevTables t;
  t.device = dev;
  size_t spad = ((size_t)s->S_dir + kRecPad - 1) / kRecPad * kRecPad;
  size_t rec_bytes = spad * s->rec_words * sizeof(uint32_t);
  e = cudaMalloc(&t.rec, rec_bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(structure records)");
  e = cudaMalloc(&t.conf_class, sizeof(int32_t) * (size_t)s->S_dir);
  if (e != cudaSuccess) {
    cudaFree(t.rec);
    return cuda_fail(e, "cudaMalloc(class table)");
  }
  // synchronous upload on the legacy stream: happens once per library and device
  e = cudaMemset(t.rec, 0, rec_bytes);
  if (e == cudaSuccess)
    e = cudaMemcpy(t.rec, s->rec.data(), s->rec.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(t.conf_class, s->conf_class.data(), sizeof(int32_t) * (size_t)s->S_dir,
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(t.rec);
    cudaFree(t.conf_class);
    return cuda_fail(e, "upload of structure tables");
  }
  DevTables* keep = new (std::nothrow) DevTables(t);
  if (!keep) {
    cudaFree(t.rec);
    cudaFree(t.conf_class);
    return fail(HP_ENOMEM, "device table bookkeeping: out of host memory");
  }
  s->dev.push_back(keep);
  *out = keep;
  return HP_OK;
}

}  // namespace hp

extern "C" const char* hp_last_error(void) { return g_last_error.c_str(); }

extern "C" int hp_set_wait_limit(int64_t polls) {
  g_wait_limit.store(polls < 0 ? -1 : (long long)polls, std::memory_order_relaxed);
  return HP_OK;
}

extern "C" void hp_structs_free(hp_structs* s) {
  if (!s) return;
  int cur = -1;
  cudaGetDevice(&cur);
  for (hp::DevTables* t : s->dev) {
    if (cudaSetDevice(t->device) == cudaSuccess) {
      cudaFree(t->rec);
      cudaFree(t->conf_class);
      if (t->scan_gcnt) cudaFree(t->scan_gcnt);
      if (t->scan_ccnt) cudaFree(t->scan_ccnt);
      if (t->scan_cl1) cudaFree(t->scan_cl1);
      if (t->scan_gbeg) cudaFree(t->scan_gbeg);
      if (t->scan_mcnt) cudaFree(t->scan_mcnt);
      if (t->scan_mmask) cudaFree(t->scan_mmask);
      if (t->scan_midx) cudaFree(t->scan_midx);
      if (t->class_first) cudaFree(t->class_first);
      if (t->class_nconf) cudaFree(t->class_nconf);
      if (t->half_otab) cudaFree(t->half_otab);
    }
    delete t;
  }
  if (cur >= 0 && !s->dev.empty()) cudaSetDevice(cur);
  delete s;
}
