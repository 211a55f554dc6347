// tdct_search.h -- GPU greedy angle search (internal interface).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace tdct {

constexpr int kSearchMaxN = 16;
constexpr double kSearchTieTol = 1e-12;
constexpr int kSearchMaxAbs = 16;  // alphabet values lie in [-16, 16]
constexpr int kSearchHitCap = 65536;  // hit list entries allocated

struct SearchParams {
  double crow_rev[kSearchMaxN];         // exact DCT row, coordinates reversed, zero past N
  int32_t alphabet[9];                  // sorted, distinct
  int32_t np;                           // alphabet size
  int32_t N;
  uint32_t total;                       // np^N candidates (zero vector included)
  int32_t n_fixed;
  int32_t tie_large;                    // 0: smaller norm first, 1: larger
  int32_t max_n2;                       // N * max(v^2): largest squared norm
  int32_t hit_cap;                      // hit list capacity, <= kSearchHitCap
  int8_t fixed[kSearchMaxN][kSearchMaxN];  // preset rows (coordinate order)
};

struct SearchState {
  unsigned long long best_key;  // order-preserving key of the best FP64 cosine (0 = none yet)
  unsigned long long pick_key;  // (norm key << 32) | index of the winner (~0 = none yet)
  uint32_t best32;              // order-preserving key of the best FP32 cosine (0 = none yet)
  uint32_t n_hits;              // screened candidates this row (list overflowed if > cap)
  int32_t dead;                 // a row had no allowed candidate
  int32_t n_done;               // rows committed so far
  int8_t last_row[kSearchMaxN];
  uint32_t chosen[kSearchMaxN];  // winner index per searched row
};

// A candidate that passed the FP32 screen, with its FP64 cosine.
struct SearchHit {
  uint32_t i;
  int32_t n2;
  double cosv;
};

// Enqueue the launches of one searched row.  `first`: build the allowed
// mask (one byte per candidate) from the presets; later rows test against
// the row chosen last and clear the mask of the candidates it rejects.
cudaError_t enqueue_search_row(const SearchParams& sp, SearchState* st, uint8_t* allowed,
                               SearchHit* hits, int first, int slot, cudaStream_t s);

}  // namespace tdct
