// batch_types.cuh -- the work description of the batched iteration (many
// independent VEGAS integrations per launch, the loop of Sec. 2.1 for every
// instance), shared by the batched sampling kernels and their host code.
#pragma once

#include "common.cuh"

namespace gv {

constexpr int kBatchHist = 64;   // iterations kept per instance
constexpr int kBatchDM = 16;     // compile-time dimension bound
constexpr int kRowTail = 3;      // sum w, sum w^2, non-finite count

struct BatchInst {
  int kind, d, first_item, nitems;
  uint64_t ncall;
  uint32_t instance;
  int tab_off;    // cells: [d][N] in tab64 / tab32
  int edge_off;   // [d][N+1] in edges
  int bins_off;   // [2][d][N] in bins
  double alpha;
};

struct BatchItem {
  int inst;
  uint32_t s0, count;
  uint32_t row;   // offset of the item's partial row (2 d N + kRowTail entries)
};

struct BatchState {
  uint32_t it;
  int nhist;
  long long nonfinite, samples;
  double I, sigma, chi2, last_I, last_var;
  double hist[kBatchHist][2];
};

struct BatchArgs {
  int n, nitems, N, cap, ppt;
  int maxd;  // widest instance (the general kernel's shared-memory layout)
  uint32_t key0, key1;
  uint32_t ks[kPhiloxKeyWords];  // Philox round keys of (key0, key1)
  const BatchInst* inst;
  const BatchItem* items;
  const void* tab;        // float2 (FP32 form) or double2 (FP64) cells
  const double* dparams;  // [n][kNumDerived]
  int* head;              // next item
  void* rows;             // float2 pairs (FP32 form) or doubles
  BatchState* st;
  double* edges;
  double2* tab64;
  float2* tab32;
  double* bins;
  const int2* axis_map;   // finalisation block -> (instance, axis)
  int naxes, refine, record, pair32;
};

// Items of one dimension kernel's queue (the FP32 form with 24-bit words).
struct BatchRange {
  int first, count;  // items [first, first + count) of this dimension
  int* head;         // its queue counter
  int cap;           // bucket capacity (slots per bucket row)
};

}  // namespace gv
