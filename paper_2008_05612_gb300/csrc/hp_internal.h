// Internal declarations shared by the translation units of libhp_gpmap.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hp_gpmap.h"

namespace hp {

constexpr int kMaxN = 40;       // residues per chain
constexpr int kMaxHalf = 20;    // even (or odd) residues per chain
constexpr int kMaxSym = 48;     // order of the cube's symmetry group

// Sets the thread-local error text and returns `code`.
int fail(int code, const std::string& msg);
int cuda_fail(int err, const char* what);  // err is a cudaError_t

// Per-device copy of a fold library's kernel tables.
struct DevTables {
  int device = -1;
  uint32_t* rec = nullptr;       // S_pad x rec_words contact records
  int32_t* conf_class = nullptr; // S_dir class ids
  // per-sequence scan tables (built on first use): conformations sorted by their contact-count
  // vectors; a group is a run of equal vectors (equal A for every sequence)
  uint32_t* scan_gcnt = nullptr;   // 6 x gpad: per group the six count bit-planes, word-major
  uint32_t* scan_ccnt = nullptr;   // 12 x cpad: per cluster of groups the planes of the minimum and excess
  int32_t* scan_cl1 = nullptr;     // cpad: per cluster the largest L1 excess
  int32_t* scan_gbeg = nullptr;    // ngroups + 1: first member of each group (scan order)
  uint32_t* scan_mcnt = nullptr;   // 6 x spad: per member its count bit-planes, word-major
  uint32_t* scan_mmask = nullptr;  // NE x spad: per member its contact masks, word-major
  int32_t* scan_midx = nullptr;    // spad: original conformation index of each member
  int scan_ngroups = 0, scan_gpad = 0, scan_spad = 0, scan_cpad = 0;
  // class -> first conformation index and number of conformations (built on first use)
  int32_t* class_first = nullptr;
  int32_t* class_nconf = nullptr;
  // odd-residue patterns o with o <= reverse(o) (odd N only; built on first use)
  uint32_t* half_otab = nullptr;
  int half_n = 0;
};

}  // namespace hp

// Fold library (opaque in the C ABI).
struct hp_structs {
  int ndim = 0;
  int L[3] = {1, 1, 1};
  int N = 0;
  int NE = 0;        // even residues: 0, 2, 4, ...
  int NO = 0;        // odd residues: 1, 3, 5, ...
  int C = 0;         // contacts per conformation
  int nsym = 0;
  int32_t S = 0;     // classes
  int32_t S_dir = 0; // directed conformations
  std::vector<uint8_t> conf;        // S_dir x N sites
  std::vector<int32_t> conf_class;  // S_dir
  std::vector<uint8_t> contacts;    // S_dir x C x 2 residues (i < j)
  // Kernel record of each conformation (rec_words uint32, rec_words odd so a
  // thread-per-record shared-memory read is conflict-free):
  //   [k]      for k < NE: contact mask of even residue 2k over odd residues
  //            (bit j = odd residue 2j+1)
  //   [NE+b]   for b < 3: bit b of the contact count of each odd residue,
  //            as a mask over odd residues
  //   [NE+3+b] for b < 3: bit b of the contact count of each even residue,
  //            as a mask over even residues (bit k = residue 2k)
  //   rest     zero padding
  int rec_words = 0;
  std::vector<uint32_t> rec;        // S_dir x rec_words
  int tile_reg_bits = 0;            // preferred kernel shape (0: library default), see hp_set_tile_cfg
  int tile_size = 0;
  std::mutex mu;
  std::vector<hp::DevTables*> dev;  // lazily uploaded, one entry per device
};

namespace hp {
// Upload (once per device) and return the device tables for the current device.
int device_tables(const hp_structs* s, DevTables** out);
// Same, plus the per-sequence scan tables.
int scan_tables(const hp_structs* s, DevTables** out);
// Same, plus the table of reversal-canonical odd patterns (odd N).
int half_tables(const hp_structs* s, DevTables** out);
// Records are padded on the device to a multiple of this many conformations.
constexpr int kRecPad = 256;
// Poll limit for the bounded device-side waits of the kernels: `dflt` (the kernel's own
// constant) unless hp_set_wait_limit has set a limit for this process.
long long wait_limit(long long dflt);
// Eq. 2 numerators of a full 2^N map (robustness tile pass): ADDS to neutral / to_del [S + 1] and
// counts the -1 genotypes into *negcount (all caller-zeroed); error bits go to *err.
cudaError_t launch_robustness(const int32_t* d_phen, int N, int S, unsigned long long* neutral,
                              unsigned long long* to_del, unsigned long long* negcount, unsigned* err, cudaStream_t st);
}  // namespace hp
