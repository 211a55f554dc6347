// tdct_search.cu -- the greedy angle search of §3 (Eq. (6); §6.2 poses it for
// N = 16) on the GPU, for one row order.
//
// Candidates are the |P|^N vectors over an alphabet P, enumerated as base-|P|
// numbers over the sorted alphabet with the first coordinate most
// significant; the zero vector is not a candidate.  For each row k of the
// order, in turn:
//   t_k = argmax cos(c_k, d) = <c_k, d> / ||d||   over candidates d orthogonal
//         to every row chosen (or preset) so far,
// with values within 1e-12 of the maximum counted as ties, decided by the
// norm (smaller or larger first) and then by the enumeration index.
//
// Per row, three launches:
//   max pass:  every candidate still allowed is tested against the row chosen
//              last (the presets on the first pass); survivors get their FP64
//              cosine written to `cosv` (rejected ones -inf, permanently), and
//              the maximum goes to an order-preserving 64-bit key (atomicMax);
//   pick pass: candidates within the tolerance of the maximum compete on
//              (norm key << 32 | index) (atomicMin);
//   commit:    one thread decodes the winner and records it (or a dead end).
#include <cuda_runtime.h>

#include <cstdint>

#include "tdct_search.h"

namespace tdct {

namespace {

__device__ __forceinline__ unsigned long long order_key(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

// Digits of candidate `idx`, least significant first: d[k] is coordinate
// N - 1 - k.  Digits beyond N are left 0 and masked by the callers.
template <int NP>
__device__ __forceinline__ void decode(uint32_t idx, int N, const SearchParams& sp,
                                       int (&v)[kSearchMaxN]) {
#pragma unroll
  for (int k = 0; k < kSearchMaxN; ++k) {
    const uint32_t q = idx / NP, dgt = idx - q * NP;
    v[k] = k < N ? sp.alphabet[dgt] : 0;
    idx = q;
  }
}

template <int NP>
__global__ void __launch_bounds__(256) search_max(SearchParams sp, SearchState* __restrict__ st,
                                                  double* __restrict__ cosv, int first) {
  if (st->dead) return;
  __shared__ int8_t against[kSearchMaxN][kSearchMaxN];  // reversed rows to test against
  __shared__ int n_against;
  __shared__ unsigned long long warp_best[8];
  if (threadIdx.x == 0) n_against = first ? sp.n_fixed : 1;
  for (int e = threadIdx.x; e < kSearchMaxN * kSearchMaxN; e += blockDim.x) {
    const int r = e / kSearchMaxN, k = e % kSearchMaxN;
    int8_t val = 0;
    if (k < sp.N) {
      if (first) val = r < sp.n_fixed ? sp.fixed[r][sp.N - 1 - k] : 0;
      else val = r == 0 ? st->last_row[sp.N - 1 - k] : 0;
    }
    against[r][k] = val;
  }
  __syncthreads();
  const int nag = n_against;
  unsigned long long best = 0ull;  // below every key of a finite value
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < sp.total;
       i += gridDim.x * blockDim.x) {
    if (!first && cosv[i] == -INFINITY) continue;
    int v[kSearchMaxN];
    decode<NP>(i, sp.N, sp, v);
    int n2 = 0;
#pragma unroll
    for (int k = 0; k < kSearchMaxN; ++k) n2 += v[k] * v[k];
    bool ok = n2 > 0;
    for (int r = 0; r < nag && ok; ++r) {
      int dot = 0;
#pragma unroll
      for (int k = 0; k < kSearchMaxN; ++k) dot += v[k] * against[r][k];
      ok = dot == 0;
    }
    double c = -INFINITY;
    if (ok) {
      double dot = 0.0;
#pragma unroll
      for (int k = 0; k < kSearchMaxN; ++k) dot = fma(sp.crow_rev[k], (double)v[k], dot);
      c = dot / sqrt((double)n2);
      const unsigned long long key = order_key(c);
      best = key > best ? key : best;
    }
    cosv[i] = c;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_down_sync(0xffffffffu, best, o);
    best = other > best ? other : best;
  }
  if ((threadIdx.x & 31) == 0) warp_best[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = 0ull;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = warp_best[w] > b ? warp_best[w] : b;
    if (b) atomicMax(&st->best_key, b);
  }
}

template <int NP>
__global__ void __launch_bounds__(256) search_pick(SearchParams sp, SearchState* __restrict__ st,
                                                   const double* __restrict__ cosv) {
  if (st->dead || st->best_key == 0ull) return;
  const double lim = key_value(st->best_key) - kSearchTieTol;
  unsigned long long pick = ~0ull;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < sp.total;
       i += gridDim.x * blockDim.x) {
    if (!(cosv[i] >= lim)) continue;
    int v[kSearchMaxN];
    decode<NP>(i, sp.N, sp, v);
    int n2 = 0;
#pragma unroll
    for (int k = 0; k < kSearchMaxN; ++k) n2 += v[k] * v[k];
    const unsigned long long nk = sp.tie_large ? (unsigned long long)(0xffffff - n2)
                                               : (unsigned long long)n2;
    const unsigned long long key = (nk << 32) | i;
    pick = key < pick ? key : pick;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_down_sync(0xffffffffu, pick, o);
    pick = other < pick ? other : pick;
  }
  if ((threadIdx.x & 31) == 0 && pick != ~0ull) atomicMin(&st->pick_key, pick);
}

template <int NP>
__global__ void search_commit(SearchParams sp, SearchState* __restrict__ st, int slot) {
  if (st->dead) return;
  if (st->best_key == 0ull || st->pick_key == ~0ull) {
    st->dead = 1;
    return;
  }
  const uint32_t idx = (uint32_t)(st->pick_key & 0xffffffffull);
  st->chosen[slot] = idx;
  int v[kSearchMaxN];
  decode<NP>(idx, sp.N, sp, v);
#pragma unroll
  for (int k = 0; k < kSearchMaxN; ++k)
    if (k < sp.N) st->last_row[sp.N - 1 - k] = (int8_t)v[k];
  st->n_done = slot + 1;
  st->best_key = 0ull;
  st->pick_key = ~0ull;
}

template <int NP>
cudaError_t enqueue_row(const SearchParams& sp, SearchState* st, double* cosv, int first,
                        int slot, int grid, cudaStream_t s) {
  search_max<NP><<<grid, 256, 0, s>>>(sp, st, cosv, first);
  search_pick<NP><<<grid, 256, 0, s>>>(sp, st, cosv);
  search_commit<NP><<<1, 1, 0, s>>>(sp, st, slot);
  return cudaGetLastError();
}

}  // namespace

cudaError_t enqueue_search_row(const SearchParams& sp, SearchState* st, double* cosv, int first,
                               int slot, cudaStream_t s) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = ((int64_t)sp.total + 255) / 256;
  if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
  if (grid < 1) grid = 1;
  switch (sp.np) {
    case 2: return enqueue_row<2>(sp, st, cosv, first, slot, (int)grid, s);
    case 3: return enqueue_row<3>(sp, st, cosv, first, slot, (int)grid, s);
    case 4: return enqueue_row<4>(sp, st, cosv, first, slot, (int)grid, s);
    case 5: return enqueue_row<5>(sp, st, cosv, first, slot, (int)grid, s);
    case 6: return enqueue_row<6>(sp, st, cosv, first, slot, (int)grid, s);
    case 7: return enqueue_row<7>(sp, st, cosv, first, slot, (int)grid, s);
    case 8: return enqueue_row<8>(sp, st, cosv, first, slot, (int)grid, s);
    case 9: return enqueue_row<9>(sp, st, cosv, first, slot, (int)grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tdct
