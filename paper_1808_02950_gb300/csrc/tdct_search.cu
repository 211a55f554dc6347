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
// Per row:
//   max32:  candidates still allowed (a byte mask) are tested against the row
//           chosen last (rejections clear the mask for good); survivors get an
//           FP32 cosine from per-group tables and the FP32 maximum is kept;
//   max64:  candidates within kScreen of the FP32 maximum get the FP64
//           cosine; the FP64 maximum is kept (order-preserving atomicMax)
//           and the screened candidates go to a small hit list;
//   pick:   the screened candidates within the 1e-12 tolerance of the FP64
//           maximum compete on (norm key << 32 | index) (atomicMin), read
//           from the hit list (a full rescan only if the list overflowed);
//   commit: one thread decodes the winner and records it (or a dead end).
// A candidate is the sum of its digit groups' table entries (groups of 4
// digits, 3 for |P| >= 8): FP32 and FP64 partial dot products with the exact
// DCT row, partial squared norms and partial dot products with the row
// chosen last.  Presets are applied to the mask by filter passes first.
//
// Screening loses no candidate: the group partial products satisfy
// sum |<c_g, d_g>| <= ||c|| ||d|| = ||d||, so the FP32 cosine (at most six
// rounded table entries, five additions, one multiplication by a rounded
// 1 / sqrt(n2)) is within 9 * 2^-24 < 5.4e-7 of the true one.  Every
// candidate within the tie tolerance of the true maximum therefore lies
// within 1.1e-6 + 1e-12 of the FP32 maximum, well inside kScreen = 1e-5.
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

constexpr float kScreen = 1e-5f;

__device__ __forceinline__ uint32_t order_key32(float v) {
  const uint32_t b = __float_as_uint(v);
  return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_value32(uint32_t k) {
  return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k);
}

// Shared-memory tables of one pass, laid out after the 1/sqrt(n2) tables.
struct Tables {
  const double* inv64;
  const float* inv32;
  const double* d64;
  const float* d32;
  const int* n2;
  const int* o;
};

template <int NP>
__device__ __forceinline__ Tables build_tables(const SearchParams& sp, const int8_t* against_rev,
                                               unsigned char* raw, int groups) {
  constexpr int G = group_digits<NP>(), E = group_entries<NP>();
  double* inv64 = reinterpret_cast<double*>(raw);
  double* d64 = inv64 + (sp.max_n2 + 1);
  float* inv32 = reinterpret_cast<float*>(d64 + groups * E);
  float* d32 = inv32 + (sp.max_n2 + 1);
  int* n2t = reinterpret_cast<int*>(d32 + groups * E);
  int* ot = n2t + groups * E;
  for (int q = threadIdx.x; q <= sp.max_n2; q += blockDim.x) {
    const double v = q > 0 ? 1.0 / sqrt((double)q) : 0.0;
    inv64[q] = v;
    inv32[q] = (float)v;
  }
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
    d64[e] = d;
    d32[e] = (float)d;
    n2t[e] = n2;
    ot[e] = o;
  }
  return Tables{inv64, inv32, d64, d32, n2t, ot};
}

// Sums over the digit groups above the lowest one (group 0), for hi = i / E.
struct Upper {
  int n2, o;
  float d32;
};

template <int NP, bool WITH_O>
__device__ __forceinline__ Upper upper_sums(uint32_t hi, int groups, const Tables& t) {
  constexpr int E = group_entries<NP>();
  Upper u{0, 0, 0.f};
  for (int g = 1; g < groups; ++g) {
    const uint32_t q = hi / E, c = hi - q * E;
    hi = q;
    u.n2 += t.n2[g * E + c];
    if (WITH_O) u.o += t.o[g * E + c];
    u.d32 += t.d32[g * E + c];
  }
  return u;
}

// One visited candidate: index, squared norm, dot product with the row
// chosen last (when asked for), FP32 dot product with the DCT row; d64()
// forms the FP64 dot product (only for the few candidates that need it).
template <int NP>
struct Cand {
  uint32_t i, hi;
  int c, groups;
  int n2, o;
  float d32;
  const Tables* t;
  __device__ __forceinline__ double d64() const {
    constexpr int E = group_entries<NP>();
    double d = t->d64[c];
    uint32_t h = hi;
    for (int g = 1; g < groups; ++g) {
      const uint32_t q = h / E, e = h - q * E;
      h = q;
      d += t->d64[g * E + e];
    }
    return d;
  }
};

// Visits the allowed candidates.  Each thread loads 16 mask bytes at a time
// and skips all-zero words (the mask is padded to whole words with zeros);
// the upper groups' sums are formed once per word (twice when the word
// crosses a group-0 boundary: E >= 16, so at most once).  f(c) returns false
// to clear the candidate's byte (written back when WRITE).
template <int NP, bool WRITE, bool WITH_O, class F>
__device__ __forceinline__ void visit_allowed(uint8_t* allowed, const SearchParams& sp, int groups,
                                              const Tables& t, F&& f) {
  constexpr int E = group_entries<NP>();
  const uint32_t words = (sp.total + 15u) / 16u;
  uint4* mw = reinterpret_cast<uint4*>(allowed);
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < words;
       w += gridDim.x * blockDim.x) {
    const uint4 m = mw[w];
    uint32_t part[4] = {m.x, m.y, m.z, m.w};
    if ((part[0] | part[1] | part[2] | part[3]) == 0u) continue;
    const uint32_t base = w * 16u, hi = base / E;
    const int c0 = (int)(base - hi * E);
    Upper u = upper_sums<NP, WITH_O>(hi, groups, t);
    bool crossed = false, changed = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t b = part[q];
      while (b) {
        const int sh = (__ffs(b) - 1) & ~7;
        b &= ~(0xffu << sh);
        const int j = q * 4 + (sh >> 3);
        int c = c0 + j;
        if (c >= E) {  // candidates are visited in increasing order
          if (!crossed) {
            u = upper_sums<NP, WITH_O>(hi + 1, groups, t);
            crossed = true;
          }
          c -= E;
        }
        Cand<NP> cd;
        cd.i = base + (uint32_t)j;
        cd.hi = crossed ? hi + 1 : hi;
        cd.c = c;
        cd.groups = groups;
        cd.n2 = u.n2 + t.n2[c];
        cd.o = WITH_O ? u.o + t.o[c] : 0;
        cd.d32 = u.d32 + t.d32[c];
        cd.t = &t;
        if (!f(cd)) {
          part[q] &= ~(0xffu << sh);
          changed = true;
        }
      }
    }
    if (WRITE && changed) mw[w] = make_uint4(part[0], part[1], part[2], part[3]);
  }
}

// Mask initialisation (init: allowed = nonzero, padding bytes zero) and
// presets (allowed candidates not orthogonal to preset row `preset` are
// cleared).
template <int NP>
__global__ void __launch_bounds__(256) search_filter(SearchParams sp, uint8_t* __restrict__ allowed,
                                                     int preset, int init) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int G = group_digits<NP>(), E = group_entries<NP>();
  const int groups = (sp.N + G - 1) / G;
  __shared__ int8_t rev[kSearchMaxN];
  if (threadIdx.x < kSearchMaxN)
    rev[threadIdx.x] =
        (preset >= 0 && (int)threadIdx.x < sp.N) ? sp.fixed[preset][sp.N - 1 - threadIdx.x] : 0;
  __syncthreads();
  const Tables t = build_tables<NP>(sp, rev, smem_raw, groups);
  __syncthreads();
  if (init) {
    const uint32_t words = (sp.total + 15u) / 16u;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < words;
         w += gridDim.x * blockDim.x) {
      const uint32_t base = w * 16u, hi = base / E;
      const int c0 = (int)(base - hi * E);
      const int n2a = upper_sums<NP, false>(hi, groups, t).n2;
      const int n2b = upper_sums<NP, false>(hi + 1, groups, t).n2;
      uint32_t part[4] = {0u, 0u, 0u, 0u};
      for (int j = 0; j < 16; ++j) {
        if (base + (uint32_t)j >= sp.total) break;
        const int c = c0 + j;
        const int n2 = c < E ? n2a + t.n2[c] : n2b + t.n2[c - E];
        if (n2 > 0) part[j >> 2] |= 1u << ((j & 3) * 8);
      }
      reinterpret_cast<uint4*>(allowed)[w] = make_uint4(part[0], part[1], part[2], part[3]);
    }
    return;
  }
  visit_allowed<NP, true, true>(allowed, sp, groups, t,
                                [&](const Cand<NP>& c) { return c.o == 0; });
}

template <int NP>
__global__ void __launch_bounds__(256) search_max32(SearchParams sp, SearchState* __restrict__ st,
                                                    uint8_t* __restrict__ allowed, int first) {
  if (st->dead) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int G = group_digits<NP>();
  const int groups = (sp.N + G - 1) / G;
  __shared__ int8_t rev[kSearchMaxN];
  __shared__ uint32_t warp_best[8];
  if (threadIdx.x < kSearchMaxN)
    rev[threadIdx.x] = (!first && (int)threadIdx.x < sp.N) ? st->last_row[sp.N - 1 - threadIdx.x] : 0;
  __syncthreads();
  const Tables t = build_tables<NP>(sp, first ? nullptr : rev, smem_raw, groups);
  __syncthreads();
  uint32_t best = 0u;
  visit_allowed<NP, true, true>(allowed, sp, groups, t, [&](const Cand<NP>& c) {
    if (c.o != 0) return false;  // not orthogonal to the row chosen last: rejected for good
    const uint32_t key = order_key32(c.d32 * t.inv32[c.n2]);
    best = key > best ? key : best;
    return true;
  });
  for (int off = 16; off > 0; off >>= 1) {
    const uint32_t other = __shfl_down_sync(0xffffffffu, best, off);
    best = other > best ? other : best;
  }
  if ((threadIdx.x & 31) == 0) warp_best[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t b = 0u;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = warp_best[w] > b ? warp_best[w] : b;
    if (b) atomicMax(&st->best32, b);
  }
}

// FP64 maximum over the screened candidates; each is also written to the
// hit list (while it has room) so that the pick pass can skip the scan.
template <int NP>
__global__ void __launch_bounds__(256) search_max64(SearchParams sp, SearchState* __restrict__ st,
                                                    uint8_t* __restrict__ allowed,
                                                    SearchHit* __restrict__ hits) {
  if (st->dead || st->best32 == 0u) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int G = group_digits<NP>();
  const int groups = (sp.N + G - 1) / G;
  __shared__ unsigned long long warp_best[8];
  const Tables t = build_tables<NP>(sp, nullptr, smem_raw, groups);
  __syncthreads();
  const float lim32 = key_value32(st->best32) - kScreen;
  unsigned long long best = 0ull;
  visit_allowed<NP, false, false>(allowed, sp, groups, t, [&](const Cand<NP>& c) {
    if (c.d32 * t.inv32[c.n2] >= lim32) {
      const double cosv = c.d64() * t.inv64[c.n2];
      const unsigned long long key = order_key(cosv);
      best = key > best ? key : best;
      const uint32_t slot = atomicAdd(&st->n_hits, 1u);
      if (slot < (uint32_t)sp.hit_cap) hits[slot] = SearchHit{c.i, c.n2, cosv};
    }
    return true;
  });
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long other = __shfl_down_sync(0xffffffffu, best, off);
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

// Winner among the candidates within the tie tolerance of the FP64 maximum:
// block 0 reads the hit list, or, when the list overflowed, every block
// scans again with the same screen.
template <int NP>
__global__ void __launch_bounds__(256) search_pick(SearchParams sp, SearchState* __restrict__ st,
                                                   uint8_t* __restrict__ allowed,
                                                   const SearchHit* __restrict__ hits) {
  if (st->dead || st->best_key == 0ull) return;
  const uint32_t n_hits = st->n_hits;
  const bool from_list = n_hits <= (uint32_t)sp.hit_cap;
  if (from_list && blockIdx.x != 0) return;
  const double lim64 = key_value(st->best_key) - kSearchTieTol;
  unsigned long long pick = ~0ull;
  auto consider = [&](uint32_t i, int n2) {
    const unsigned long long nk = sp.tie_large ? (unsigned long long)(0xffffff - n2)
                                               : (unsigned long long)n2;
    const unsigned long long key = (nk << 32) | i;
    pick = key < pick ? key : pick;
  };
  if (from_list) {
    for (uint32_t h = threadIdx.x; h < n_hits; h += blockDim.x)
      if (hits[h].cosv >= lim64) consider(hits[h].i, hits[h].n2);
  } else {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int G = group_digits<NP>();
    const int groups = (sp.N + G - 1) / G;
    const Tables t = build_tables<NP>(sp, nullptr, smem_raw, groups);
    __syncthreads();
    const float lim32 = key_value32(st->best32) - kScreen;
    visit_allowed<NP, false, false>(allowed, sp, groups, t, [&](const Cand<NP>& c) {
      if (c.d32 * t.inv32[c.n2] >= lim32 && c.d64() * t.inv64[c.n2] >= lim64) consider(c.i, c.n2);
      return true;
    });
  }
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long other = __shfl_down_sync(0xffffffffu, pick, off);
    pick = other < pick ? other : pick;
  }
  if ((threadIdx.x & 31) == 0 && pick != ~0ull) atomicMin(&st->pick_key, pick);
}

template <int NP>
__global__ void search_commit(SearchParams sp, SearchState* __restrict__ st, int slot) {
  if (st->dead) return;
  if (st->best32 == 0u || st->best_key == 0ull || st->pick_key == ~0ull) {
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
  st->best32 = 0u;
  st->best_key = 0ull;
  st->pick_key = ~0ull;
  st->n_hits = 0u;
}

constexpr int kSearchMaxSmem = 200 * 1024;

template <int NP>
size_t table_bytes(const SearchParams& sp) {
  constexpr int G = group_digits<NP>();
  return (size_t)(sp.max_n2 + 1) * 12 +
         (size_t)((sp.N + G - 1) / G) * group_entries<NP>() * 20;
}

template <int NP>
cudaError_t enqueue_row(const SearchParams& sp, SearchState* st, uint8_t* allowed, SearchHit* hits,
                        int first, int slot, int grid, cudaStream_t s) {
  const size_t smem = table_bytes<NP>(sp);
  if (smem > (size_t)kSearchMaxSmem) return cudaErrorInvalidValue;
  // the opt-in shared-memory limit is raised once per instantiation
  static int limit_set = 0;
  if (!limit_set) {
    cudaError_t e = cudaSuccess;
    for (const void* f : {(const void*)search_filter<NP>, (const void*)search_max32<NP>,
                          (const void*)search_max64<NP>, (const void*)search_pick<NP>})
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kSearchMaxSmem);
    if (e != cudaSuccess) return e;
    limit_set = 1;
  }
  if (first) {
    search_filter<NP><<<grid, 256, smem, s>>>(sp, allowed, -1, 1);
    for (int f = 0; f < sp.n_fixed; ++f) search_filter<NP><<<grid, 256, smem, s>>>(sp, allowed, f, 0);
  }
  search_max32<NP><<<grid, 256, smem, s>>>(sp, st, allowed, first);
  search_max64<NP><<<grid, 256, smem, s>>>(sp, st, allowed, hits);
  search_pick<NP><<<grid, 256, smem, s>>>(sp, st, allowed, hits);
  search_commit<NP><<<1, 1, 0, s>>>(sp, st, slot);
  return cudaGetLastError();
}

}  // namespace

cudaError_t enqueue_search_row(const SearchParams& sp, SearchState* st, uint8_t* allowed,
                               SearchHit* hits, int first, int slot, cudaStream_t s) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = ((int64_t)sp.total + 16 * 256 - 1) / (16 * 256);  // 16 candidates per thread
  if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
  if (grid < 1) grid = 1;
  switch (sp.np) {
    case 2: return enqueue_row<2>(sp, st, allowed, hits, first, slot, (int)grid, s);
    case 3: return enqueue_row<3>(sp, st, allowed, hits, first, slot, (int)grid, s);
    case 4: return enqueue_row<4>(sp, st, allowed, hits, first, slot, (int)grid, s);
    case 5: return enqueue_row<5>(sp, st, allowed, hits, first, slot, (int)grid, s);
    case 6: return enqueue_row<6>(sp, st, allowed, hits, first, slot, (int)grid, s);
    case 7: return enqueue_row<7>(sp, st, allowed, hits, first, slot, (int)grid, s);
    case 8: return enqueue_row<8>(sp, st, allowed, hits, first, slot, (int)grid, s);
    case 9: return enqueue_row<9>(sp, st, allowed, hits, first, slot, (int)grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tdct
