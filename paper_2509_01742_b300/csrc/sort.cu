// sort.cu -- bitonic sorting network for the oblivious build and the batch
// grouping step.
//
// The network is the standard ascending bitonic sort on a power-of-two array:
// stage s (s = 1..log2 n) merges runs of 2^s; its steps compare element i with
// i | 2^b for b = s-1 down to 0, ascending where bit s of i is 0 and
// descending where it is 1.  Which pairs are compared never depends on the
// data, so the memory access pattern is fixed (the build's "oblivious sort").
//
// B300 mapping:
//   - tile kernel: a CTA owns 2^LT consecutive elements in shared memory (one
//     pad word per 16 elements keeps 8- and 16-byte accesses free of bank
//     conflicts) and runs every step with stride < 2^LT; each thread holds 16
//     elements in registers, so four consecutive stride bits are handled per
//     shared-memory round trip instead of one;
//   - global kernel: steps with stride >= 2^LT, up to four consecutive stride
//     bits fused per HBM pass; each thread keeps 2 x 2^nb elements in
//     registers and reads/writes them as 16-byte vectors, so every warp access
//     is a fully coalesced 512-byte segment.
#include "bolt_internal.cuh"
#include "batch.cuh"

namespace bdev {

struct KeyU64 {
  static __device__ __forceinline__ bool less(uint64_t a, uint64_t b) { return a < b; }
};
struct KeyPair {
  static __device__ __forceinline__ bool less(const ulonglong2& a, const ulonglong2& b) {
    return a.x < b.x || (a.x == b.x && a.y < b.y);
  }
};

template <typename T, typename Cmp>
__device__ __forceinline__ void cmp_swap(T& a, T& b, bool ascending) {
  // keep (min, max) when ascending, (max, min) when descending
  bool swap = ascending ? Cmp::less(b, a) : Cmp::less(a, b);
  if (swap) {
    T t = a;
    a = b;
    b = t;
  }
}

__device__ __forceinline__ uint32_t pad_idx(uint32_t i) { return i + (i >> 4); }

// Insert the 4-bit register index r at bit position w_lo of the thread's
// remaining index bits t.
__device__ __forceinline__ uint32_t spread4(uint32_t t, uint32_t r, int w_lo) {
  uint32_t low = t & ((1u << w_lo) - 1u);
  uint32_t high = t >> w_lo;
  return (high << (w_lo + 4)) | (r << w_lo) | low;
}

// Run steps b = b_hi .. b_lo of stage s on the tile held in shared memory.
// All bits are < LT.  The 4-bit register window [w_lo, w_lo + 3] covers them.
template <typename T, typename Cmp, int LT>
__device__ __forceinline__ void tile_round(T* sm, uint64_t tile_base, int s, int b_hi, int b_lo) {
  const int w_lo = b_lo <= LT - 4 ? b_lo : LT - 4;
  const uint32_t t = threadIdx.x;
  T v[16];
#pragma unroll
  for (int r = 0; r < 16; r++) v[r] = sm[pad_idx(spread4(t, r, w_lo))];
#pragma unroll
  for (int rb = 3; rb >= 0; rb--) {  // register bit rb is stride bit w_lo + rb
    const int b = w_lo + rb;
    if (b > b_hi || b < b_lo) continue;
#pragma unroll
    for (int r = 0; r < 16; r++) {
      if (r & (1 << rb)) continue;
      const uint64_t gi = tile_base + spread4(t, r, w_lo);
      const bool asc = ((gi >> s) & 1) == 0;
      cmp_swap<T, Cmp>(v[r], v[r | (1 << rb)], asc);
    }
  }
#pragma unroll
  for (int r = 0; r < 16; r++) sm[pad_idx(spread4(t, r, w_lo))] = v[r];
}

// full = 1: stages 1..LT of the tile (sorts the tile into alternating
// directions); full = 0: the in-tile steps (bits LT-1..0) of stage s > LT.
template <typename T, typename Cmp, int LT>
__global__ void __launch_bounds__((1 << LT) / 16) k_sort_tile(T* data, int s_merge, int full) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  constexpr uint32_t TILE = 1u << LT;
  constexpr uint32_t NT = TILE / 16;
  const uint64_t base = (uint64_t)blockIdx.x * TILE;
  for (uint32_t i = threadIdx.x; i < TILE; i += NT) sm[pad_idx(i)] = data[base + i];
  __syncthreads();
  if (full) {
    for (int s = 1; s <= LT; s++) {
      for (int hi = s - 1; hi >= 0; hi -= 4) {
        int lo = hi - 3 > 0 ? hi - 3 : 0;
        tile_round<T, Cmp, LT>(sm, base, s, hi, lo);
        __syncthreads();
      }
    }
  } else {
    for (int hi = LT - 1; hi >= 0; hi -= 4) {
      int lo = hi - 3 > 0 ? hi - 3 : 0;
      tile_round<T, Cmp, LT>(sm, base, s_merge, hi, lo);
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < TILE; i += NT) data[base + i] = sm[pad_idx(i)];
}

// Steps b = b_hi .. b_hi-NB+1 (all >= the tile bits) of stage s, one HBM pass.
// Thread t owns the pair of adjacent low positions (2u, 2u+1) and the 2^NB
// positions that differ in the stride bits.
template <int NB>
__global__ void __launch_bounds__(256) k_sort_global_u64(uint64_t* data, uint64_t n, int s,
                                                         int b_hi) {
  constexpr int E = 1 << NB;
  const int w_lo = b_hi - NB + 1;
  const uint64_t nthreads = n / (2 * E);
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nthreads;
       t += (uint64_t)gridDim.x * blockDim.x) {
    // t indexes pairs: low part (w_lo - 1 bits, pairs of elements) and high part
    const uint64_t low = (t << 1) & ((1ull << w_lo) - 1);
    const uint64_t high = (t << 1) >> w_lo;
    const uint64_t base = (high << (w_lo + NB)) | low;
    ulonglong2 v[E];
#pragma unroll
    for (int r = 0; r < E; r++)
      v[r] = *reinterpret_cast<const ulonglong2*>(data + (base | ((uint64_t)r << w_lo)));
    const bool asc = ((base >> s) & 1) == 0;  // bit s is above every stride bit
#pragma unroll
    for (int b = NB - 1; b >= 0; b--) {
#pragma unroll
      for (int r = 0; r < E; r++) {
        if (r & (1 << b)) continue;
        unsigned long long a0 = v[r].x, a1 = v[r].y, c0 = v[r | (1 << b)].x,
                           c1 = v[r | (1 << b)].y;
        bool sw0 = asc ? c0 < a0 : a0 < c0;
        bool sw1 = asc ? c1 < a1 : a1 < c1;
        v[r].x = sw0 ? c0 : a0;
        v[r | (1 << b)].x = sw0 ? a0 : c0;
        v[r].y = sw1 ? c1 : a1;
        v[r | (1 << b)].y = sw1 ? a1 : c1;
      }
    }
#pragma unroll
    for (int r = 0; r < E; r++)
      *reinterpret_cast<ulonglong2*>(data + (base | ((uint64_t)r << w_lo))) = v[r];
  }
}

// One step of stride 2^b (b >= tile bits) for 16-byte pairs.
__global__ void k_sort_global_pair(ulonglong2* data, uint32_t n, int s, int b) {
  uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n / 2) return;
  uint32_t low = p & ((1u << b) - 1);
  uint32_t i = ((p >> b) << (b + 1)) | low;
  uint32_t j = i | (1u << b);
  ulonglong2 a = data[i], c = data[j];
  cmp_swap<ulonglong2, KeyPair>(a, c, ((i >> s) & 1) == 0);
  data[i] = a;
  data[j] = c;
}

template <int LT, typename T>
static size_t tile_smem() {
  return (size_t)((1u << LT) + (1u << LT) / 16) * sizeof(T);
}

template <int LT>
static cudaError_t sort_u64_lt(uint64_t* tags, uint64_t n, cudaStream_t st) {
  const size_t smem = tile_smem<LT, uint64_t>();
  cudaError_t e = cudaFuncSetAttribute(k_sort_tile<uint64_t, KeyU64, LT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const uint64_t tiles = n >> LT;
  const int nt = (1 << LT) / 16;
  {
    ProfSpan ps(P_SORT_TILE, st);
    k_sort_tile<uint64_t, KeyU64, LT><<<(unsigned)tiles, nt, smem, st>>>(tags, 0, 1);
    count_launch();
  }
  int logn = 0;
  while ((1ull << logn) < n) logn++;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int s = LT + 1; s <= logn; s++) {
    for (int hi = s - 1; hi >= LT; hi -= 4) {
      int nb = hi - LT + 1 < 4 ? hi - LT + 1 : 4;
      uint64_t threads = n / (2ull << nb);
      uint64_t blocks = (threads + 255) / 256;
      uint64_t cap = (uint64_t)sms * 16;
      unsigned g = (unsigned)(blocks < cap ? blocks : cap);
      ProfSpan ps(P_SORT_GLOBAL, st);
      count_launch();
      switch (nb) {
        case 1: k_sort_global_u64<1><<<g, 256, 0, st>>>(tags, n, s, hi); break;
        case 2: k_sort_global_u64<2><<<g, 256, 0, st>>>(tags, n, s, hi); break;
        case 3: k_sort_global_u64<3><<<g, 256, 0, st>>>(tags, n, s, hi); break;
        default: k_sort_global_u64<4><<<g, 256, 0, st>>>(tags, n, s, hi); break;
      }
    }
    ProfSpan ps(P_SORT_TILE, st);
    k_sort_tile<uint64_t, KeyU64, LT><<<(unsigned)tiles, nt, smem, st>>>(tags, s, 0);
    count_launch();
  }
  return cudaGetLastError();
}

// n must be a power of two and at least 2^log_tile.
cudaError_t sort_tags_u64(uint64_t* tags, uint64_t n, int log_tile, cudaStream_t st) {
  if (n & (n - 1)) return cudaErrorInvalidValue;
  if (log_tile == 13 && n >= (1ull << 13)) return sort_u64_lt<13>(tags, n, st);
  if (log_tile == 12 && n >= (1ull << 12)) return sort_u64_lt<12>(tags, n, st);
  return cudaErrorInvalidValue;
}

// (key, payload) pairs, n a power of two: 512 (one warp, one tile) or
// 4096..65536 (4096-element tiles plus global steps).
cudaError_t sort_pairs(ulonglong2* data, uint32_t n, cudaStream_t st) {
  if (n == 512) {
    k_sort_tile<ulonglong2, KeyPair, 9><<<1, 32, tile_smem<9, ulonglong2>(), st>>>(data, 0, 1);
    count_launch();
    return cudaGetLastError();
  }
  constexpr int LT = 12;
  if (n & (n - 1) || n < (1u << LT) || n > 65536) return cudaErrorInvalidValue;
  const size_t smem = tile_smem<LT, ulonglong2>();
  cudaError_t e = cudaFuncSetAttribute(k_sort_tile<ulonglong2, KeyPair, LT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const uint32_t tiles = n >> LT;
  const int nt = (1 << LT) / 16;
  k_sort_tile<ulonglong2, KeyPair, LT><<<tiles, nt, smem, st>>>(data, 0, 1);
  count_launch();
  int logn = 0;
  while ((1u << logn) < n) logn++;
  for (int s = LT + 1; s <= logn; s++) {
    for (int b = s - 1; b >= LT; b--) {
      k_sort_global_pair<<<(n / 2 + 255) / 256, 256, 0, st>>>(data, n, s, b);
      count_launch();
    }
    k_sort_tile<ulonglong2, KeyPair, LT><<<tiles, nt, smem, st>>>(data, s, 0);
    count_launch();
  }
  return cudaGetLastError();
}

}  // namespace bdev
