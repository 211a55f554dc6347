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

// Digits per table group: NP^G entries per group stay small.
template <int NP>
__host__ __device__ constexpr int group_digits() {
  return NP <= 7 ? 4 : 3;
}
template <int NP>
__host__ __device__ constexpr int group_entries() {
  int e = 1;
  for (int t = 0; t < group_digits<NP>(); ++t) e *= NP;
  return e;
}

// Shared-memory tables of one row's pass, per group g of G digits and per
// digit combination c of that group: the FP64 partial dot product with the
// exact DCT row, the partial squared norm and the partial dot product with
// `against` (the row chosen last, or a preset).  A candidate is the sum of
// its groups' entries.
template <int NP>
__device__ __forceinline__ void build_tables(const SearchParams& sp, const int8_t* against_rev,
                                             double* dtab, int* ntab, int* otab, int groups) {
  constexpr int G = group_digits<NP>(), E = group_entries<NP>();
  for (int e = threadIdx.x; e < groups * E; e += blockDim.x) {
    const int g = e / E;
    int c = e - g * E;
    double d = 0.0;
    int n2 = 0, o = 0;
    for (int t = 0; t < G; ++t) {
      const int k = g * G + t, dg = c % NP;
      c /= NP;
      if (k < sp.N) {
        const int v = sp.alphabet[dg];
        d = fma(sp.crow_rev[k], (double)v, d);
        n2 += v * v;
        o += v * (against_rev ? against_rev[k] : 0);
      }
    }
    dtab[e] = d;
    ntab[e] = n2;
    otab[e] = o;
  }
}

// Allowed-set initialisation and presets: cosv[i] = 0 for candidates that
// are nonzero and orthogonal to the preset (or to nothing), -inf otherwise.
template <int NP>
__global__ void __launch_bounds__(256) search_filter(SearchParams sp, double* __restrict__ cosv,
                                                     int preset, int init) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int E = group_entries<NP>(), G = group_digits<NP>();
  const int groups = (sp.N + G - 1) / G;
  double* dtab = reinterpret_cast<double*>(smem_raw) + (sp.max_n2 + 1);
  int* ntab = reinterpret_cast<int*>(dtab + groups * E);
  int* otab = ntab + groups * E;
  __shared__ int8_t rev[kSearchMaxN];
  if (threadIdx.x < kSearchMaxN)
    rev[threadIdx.x] = (preset >= 0 && threadIdx.x < sp.N) ? sp.fixed[preset][sp.N - 1 - threadIdx.x] : 0;
  __syncthreads();
  build_tables<NP>(sp, rev, dtab, ntab, otab, groups);
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < sp.total;
       i += gridDim.x * blockDim.x) {
    if (!init && cosv[i] == -INFINITY) continue;
    uint32_t idx = i;
    int n2 = 0, o = 0;
    for (int g = 0; g < groups; ++g) {
      const uint32_t q = idx / E, c = idx - q * E;
      idx = q;
      n2 += ntab[g * E + c];
      o += otab[g * E + c];
    }
    const bool ok = n2 > 0 && o == 0;
    if (init || !ok) cosv[i] = ok ? 0.0 : -INFINITY;
  }
}

template <int NP>
__global__ void __launch_bounds__(256) search_max(SearchParams sp, SearchState* __restrict__ st,
                                                  double* __restrict__ cosv, int first) {
  if (st->dead) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int E = group_entries<NP>(), G = group_digits<NP>();
  const int groups = (sp.N + G - 1) / G;
  double* inv_norm = reinterpret_cast<double*>(smem_raw);  // 1 / sqrt(n2), n2 = 0..max_n2
  double* dtab = inv_norm + (sp.max_n2 + 1);
  int* ntab = reinterpret_cast<int*>(dtab + groups * E);
  int* otab = ntab + groups * E;
  __shared__ int8_t rev[kSearchMaxN];
  __shared__ unsigned long long warp_best[8];
  if (threadIdx.x < kSearchMaxN)
    rev[threadIdx.x] = (!first && threadIdx.x < sp.N) ? st->last_row[sp.N - 1 - threadIdx.x] : 0;
  for (int q = threadIdx.x; q <= sp.max_n2; q += blockDim.x)
    inv_norm[q] = q > 0 ? 1.0 / sqrt((double)q) : 0.0;
  __syncthreads();
  build_tables<NP>(sp, first ? nullptr : rev, dtab, ntab, otab, groups);
  __syncthreads();
  unsigned long long best = 0ull;  // below every key of a finite value
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < sp.total;
       i += gridDim.x * blockDim.x) {
    if (cosv[i] == -INFINITY) continue;
    uint32_t idx = i;
    int n2 = 0, o = 0;
    double dot = 0.0;
    for (int g = 0; g < groups; ++g) {
      const uint32_t q = idx / E, c = idx - q * E;
      idx = q;
      n2 += ntab[g * E + c];
      o += otab[g * E + c];
      dot += dtab[g * E + c];
    }
    double c = -INFINITY;
    if (o == 0) {  // nonzero and orthogonal to the presets: filtered before
      c = dot * inv_norm[n2];
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
size_t table_bytes(const SearchParams& sp) {
  constexpr int G = group_digits<NP>();
  return sizeof(double) * (size_t)(sp.max_n2 + 1) +
         (size_t)((sp.N + G - 1) / G) * group_entries<NP>() * (sizeof(double) + 2 * sizeof(int));
}

template <int NP>
cudaError_t enqueue_row(const SearchParams& sp, SearchState* st, double* cosv, int first,
                        int slot, int grid, cudaStream_t s) {
  const size_t smem = table_bytes<NP>(sp);
  // the opt-in shared-memory limit is raised once per instantiation, to the
  // largest table any accepted (alphabet, N) needs
  static int limit_set = 0;
  if (!limit_set) {
    constexpr int kMaxSmem = 140 * 1024;
    cudaError_t e = cudaFuncSetAttribute(search_max<NP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(search_filter<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kMaxSmem);
    if (e != cudaSuccess) return e;
    limit_set = 1;
  }
  if (smem > 140 * 1024) return cudaErrorInvalidValue;
  if (first) {
    // allowed set: nonzero candidates orthogonal to every preset
    search_filter<NP><<<grid, 256, smem, s>>>(sp, cosv, -1, 1);
    for (int f = 0; f < sp.n_fixed; ++f) search_filter<NP><<<grid, 256, smem, s>>>(sp, cosv, f, 0);
  }
  search_max<NP><<<grid, 256, smem, s>>>(sp, st, cosv, first);
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
