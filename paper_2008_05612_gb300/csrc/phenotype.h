// Launch description of the phenotype kernel (shared by the single-box,
// batched, graph-captured and autotuning entry points).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "hp_internal.h"

namespace hp {

constexpr int kPhenMaxInst = 8;      // boxes per launch
constexpr int kPhenMaxBlocks = 128;  // aligned id blocks per launch (all boxes)
constexpr size_t kPhenCtrlBytes = 16;  // [0] error word, [2..3] work counter (64-bit)

struct PhenInst {
  const uint32_t* rec;       // conformation records, padded to a multiple of the tile
  const int32_t* conf_class; // class of each conformation
  int32_t* phen;             // output, indexed by id - begin
  int32_t* aux;              // optional output (lowest-index minimiser's class)
  int S_dir, ntiles, rec_words, NE;
};

struct PhenBlock {
  unsigned long long g_base;      // first sequence id of the block (aligned to 2^m)
  unsigned long long out_off;     // output index of g_base
  unsigned long long item_begin;  // first work item of the block
  unsigned int ne_free, no_free;  // even / odd residues below bit m
  unsigned int nroles;            // real roles: min(ne_free, 14)
  unsigned int inst;              // index into PhenParams::inst
  // reversal-symmetric half enumeration (full space of an odd-length chain): the odd
  // patterns to compute (o <= reverse(o)); every result is also written at the reversed id
  const uint32_t* otab;           // NULL: every odd pattern of the block
  unsigned int ntab;              // entries of otab
  unsigned int pad;
};

struct PhenParams {
  unsigned int* ctrl;  // kPhenCtrlBytes of device memory, zeroed before each launch
  uint32_t one;        // always 1: tree additions are issued as x * one + a (IMAD)
  int ninst, nblocks, max_rec_words;
  unsigned long long total_items;
  PhenInst inst[kPhenMaxInst];
  PhenBlock blocks[kPhenMaxBlocks];
  uint32_t gap2;       // 2 x the energy-gap threshold (2: strict uniqueness, the paper's threshold 1)
  long long spin;           // polls of a bulk-copy wait before it gives up (hp_set_wait_limit)
  long long spin_handover;  // polls of a coefficient-buffer hand-over wait before it gives up
  // pass-2 work lists: wl_ctas lists of wl_stride uint16 each (2^14 entries, max ntiles + 1 offsets,
  // the listed tiles that hold candidates and their count)
  uint16_t* wlist;
  unsigned wl_stride, wl_ctas;
  int roles;  // even-pattern bits per CTA of the plan (selects the compiled shape)
};

bool tile_cfg_supported(int reg_bits, int tile);
void default_tile_cfg(int* reg_bits, int* tile);
// roles: even-pattern bits per CTA (14, or 13 / 12 / 11 for the small-role shapes)
int plan_phenotype(const hp_structs* const* libs, const uint64_t* begins, const uint64_t* counts, int n,
                   int32_t* const* d_phen, int32_t* const* d_aux, int tile, PhenParams& prm, int roles = 14);
// The compiled shape for blocks with at most max_ne_free free even residues: *roles = 14 (shape
// unchanged) or 13 / 12 / 11 with their own (reg_bits, tile).
void small_roles_shape(int max_ne_free, int* roles, int* reg_bits, int* tile);
// The role count each entry would get on its own (small_roles_shape of its blocks), into cls.
int role_classes(const hp_structs* const* libs, const uint64_t* begins, const uint64_t* counts, int n,
                 int32_t* const* d_phen, int tile, std::vector<int>& cls);
int launch_phenotype(const PhenParams& prm, int reg_bits, int tile, cudaStream_t stream, unsigned grid_limit);
// Device block a launch needs (control words, then one pass-2 work list per CTA): its size and the
// number of CTAs the launch will use; bind_launch_block points prm.ctrl / prm.wlist into it.  The
// first kPhenCtrlBytes must be zeroed before each launch.
int launch_block_bytes(const PhenParams& prm, int reg_bits, int tile, unsigned grid_limit, size_t* bytes,
                       unsigned* ctas);
void bind_launch_block(PhenParams& prm, void* block, unsigned ctas);
// plan + per-call control words + launch + error read-back (synchronises the stream); a
// gap_threshold above 1 runs the one shape compiled for it (reg_bits 5, tile 256)
// (auto_roles: use a small-role shape when every block has fewer than 14 free even residues)
int run_phenotype(const hp_structs* const* libs, const uint64_t* begins, const uint64_t* counts, int n,
                  int32_t* const* d_phen, int32_t* const* d_aux, int reg_bits, int tile, cudaStream_t st,
                  unsigned grid_limit, int gap_threshold = 1, bool auto_roles = false);

}  // namespace hp
