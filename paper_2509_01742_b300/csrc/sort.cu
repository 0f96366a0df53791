// sort.cu -- bitonic sorting network on 64-bit keys, for the oblivious build
// (page tags, key-uniqueness check) and the batch grouping step.
//
// The network is the standard ascending bitonic sort on a power-of-two array:
// stage s (s = 1..log2 n) merges runs of 2^s; its steps compare element i
// with i | 2^b for b = s-1 down to 0, keeping the smaller first where bit s of
// i is 0 and the larger first where it is 1.  Which pairs are compared never
// depends on the data, so the memory access pattern is fixed.
//
// B300 mapping:
//   - tile kernel: a CTA owns 2^LT consecutive elements.  Each thread holds 16
//     of them in registers, chosen so that 4 consecutive index bits (the
//     "window") vary across its registers; every step whose stride bit lies in
//     the window is a register compare-exchange.  Moving the window is one
//     padded shared-memory transpose (one pad word per 16 elements keeps the
//     accesses conflict-free).  Windows are compile-time, so each register's
//     address is a constant offset from a per-thread base.  Merge passes load
//     their first window straight from global memory (coalesced) and store the
//     last one straight back (16-byte vectors); the full in-tile sort loads
//     and stores 16 consecutive elements per thread as 16-byte vectors.
//   - merge passes (stage s > LT) have one direction per tile; the in-tile
//     full sort takes each pair's direction from its index bits, resolved at
//     compile time where the bit lies in the window.
//   - global kernel: steps with stride >= 2^LT, up to four consecutive stride
//     bits fused per HBM pass; each thread keeps 2 x 2^nb elements in
//     registers and moves them as 16-byte vectors.
#include "batch.cuh"
#include "bolt_internal.cuh"

namespace bdev {

template <typename T>
__device__ __forceinline__ void cx(T& a, T& b, bool asc) {
  // ascending: (min, max); descending: (max, min)
  const T lo = min(a, b), hi = max(a, b);
  a = asc ? lo : hi;
  b = asc ? hi : lo;
}

// compare-exchange with a compile-time direction
template <bool ASC, typename T>
__device__ __forceinline__ void cxd(T& a, T& b) {
  const T lo = min(a, b), hi = max(a, b);
  a = ASC ? lo : hi;
  b = ASC ? hi : lo;
}

__device__ __forceinline__ uint32_t pad_idx(uint32_t i) { return i + (i >> 4); }

// local index of register r for thread t when the window starts at bit W
template <int W>
__device__ __forceinline__ uint32_t win_idx(uint32_t t, uint32_t r) {
  return ((t >> W) << (W + 4)) | (r << W) | (t & ((1u << W) - 1u));
}

template <int W, typename T>
__device__ __forceinline__ void ld_smem(const T* sm, T v[16]) {
  const uint32_t t = threadIdx.x;
#pragma unroll
  for (int r = 0; r < 16; r++) v[r] = sm[pad_idx(win_idx<W>(t, r))];
}

template <int W, typename T>
__device__ __forceinline__ void st_smem(T* sm, const T v[16]) {
  const uint32_t t = threadIdx.x;
#pragma unroll
  for (int r = 0; r < 16; r++) sm[pad_idx(win_idx<W>(t, r))] = v[r];
}

// 16 consecutive elements per thread, moved as 16-byte vectors
template <typename T>
__device__ __forceinline__ void ld16(const T* g, T v[16]) {
  const uint4* in = reinterpret_cast<const uint4*>(g);
  constexpr int PER = 16 / sizeof(T);
#pragma unroll
  for (int k = 0; k < 16 / PER; k++) {
    const uint4 x = in[k];
    const T* e = reinterpret_cast<const T*>(&x);
#pragma unroll
    for (int j = 0; j < PER; j++) v[k * PER + j] = e[j];
  }
}

template <typename T>
__device__ __forceinline__ void st16(T* g, const T v[16]) {
  uint4* out = reinterpret_cast<uint4*>(g);
  constexpr int PER = 16 / sizeof(T);
#pragma unroll
  for (int k = 0; k < 16 / PER; k++) {
    uint4 x;
    T* e = reinterpret_cast<T*>(&x);
#pragma unroll
    for (int j = 0; j < PER; j++) e[j] = v[k * PER + j];
    out[k] = x;
  }
}

// steps for stride bits BHI..BLO (inside the window [W, W+3]), one direction
template <int W, int BHI, int BLO, bool ASC, typename T>
__device__ __forceinline__ void steps_dir(T v[16]) {
#pragma unroll
  for (int b = BHI; b >= BLO; b--) {
    const int rb = b - W;
#pragma unroll
    for (int r = 0; r < 16; r++)
      if (!(r & (1 << rb))) cxd<ASC>(v[r], v[r | (1 << rb)]);
  }
}

template <int W, int BHI, int BLO, typename T>
__device__ __forceinline__ void steps_uniform(T v[16], bool asc) {
#pragma unroll
  for (int b = BHI; b >= BLO; b--) {
    const int rb = b - W;
#pragma unroll
    for (int r = 0; r < 16; r++)
      if (!(r & (1 << rb))) cx(v[r], v[r | (1 << rb)], asc);
  }
}

// steps for stride bits BHI..BLO of stage S < LT: a pair is ascending when
// bit S of its local index is 0
template <int W, int BHI, int BLO, int S, typename T>
__device__ __forceinline__ void steps_stage(T v[16]) {
  const bool thread_asc = ((win_idx<W>(threadIdx.x, 0) >> S) & 1) == 0;
#pragma unroll
  for (int b = BHI; b >= BLO; b--) {
    const int rb = b - W;
#pragma unroll
    for (int r = 0; r < 16; r++) {
      if (r & (1 << rb)) continue;
      if (S >= W && S < W + 4) {
        if (((r >> (S - W)) & 1) == 0) cxd<true>(v[r], v[r | (1 << rb)]);
        else cxd<false>(v[r], v[r | (1 << rb)]);
      } else {
        cx(v[r], v[r | (1 << rb)], thread_asc);
      }
    }
  }
}

// window holding bits HI..LO of a chunk
template <int LT, int LO>
struct Win {
  static constexpr int value = LO <= LT - 4 ? LO : LT - 4;
};

// Merge pass, chunk of bits HI..max(HI-3,0); registers arrive in window CURW.
template <int LT, int HI, int CURW, bool ASC, typename T>
__device__ __forceinline__ void merge_chunks(T* sm, T v[16], T* gout) {
  constexpr int LO = HI - 3 > 0 ? HI - 3 : 0;
  constexpr int W = Win<LT, LO>::value;
  if constexpr (CURW != W) {
    st_smem<CURW>(sm, v);
    __syncthreads();
    ld_smem<W>(sm, v);
    __syncthreads();
  }
  steps_dir<W, HI, LO, ASC>(v);
  if constexpr (LO > 0) {
    merge_chunks<LT, LO - 1, W, ASC>(sm, v, gout);
  } else {
    static_assert(W == 0, "the last window starts at bit 0");
    // a thread's registers are 16 consecutive elements
    st16(gout + 16 * (uint64_t)threadIdx.x, v);
  }
}

// Full in-tile sort, chunk of bits HI..max(HI-3,0) of stage S; registers
// arrive in window CURW.  Stage LT's direction is the tile's (bit LT of the
// global index).
template <int LT, int S, int HI, int CURW, typename T>
__device__ __forceinline__ void full_chunks(T* sm, T v[16], bool tile_asc, T* gout) {
  constexpr int LO = HI - 3 > 0 ? HI - 3 : 0;
  constexpr int W = Win<LT, LO>::value;
  if constexpr (CURW != W) {
    st_smem<CURW>(sm, v);
    __syncthreads();
    ld_smem<W>(sm, v);
    __syncthreads();
  }
  if constexpr (S < LT) {
    steps_stage<W, HI, LO, S>(v);
  } else {
    steps_uniform<W, HI, LO>(v, tile_asc);
  }
  if constexpr (LO > 0) {
    full_chunks<LT, S, LO - 1, W>(sm, v, tile_asc, gout);
  } else if constexpr (S < LT) {
    full_chunks<LT, S + 1, S, W>(sm, v, tile_asc, gout);
  } else {
    static_assert(W == 0, "the last window starts at bit 0");
    st16(gout + 16 * (uint64_t)threadIdx.x, v);
  }
}

// Stages 1..LT of each tile (sorts tiles into alternating directions).
template <int LT, typename T>
__global__ void __launch_bounds__(1 << (LT - 4)) k_sort_tile_full(T* data) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const uint64_t base = (uint64_t)blockIdx.x << LT;
  T* g = data + base;
  T v[16];
  ld16(g + 16 * (uint64_t)threadIdx.x, v);
  full_chunks<LT, 1, 0, 0>(sm, v, ((base >> LT) & 1) == 0, g);
}

// The in-tile steps (bits LT-1..0) of stage s_merge > LT: one direction per
// tile.  Two CTAs per SM overlap one tile's loads with another's compute.
template <int LT, typename T>
__global__ void __launch_bounds__(1 << (LT - 4), 2) k_sort_tile_merge(T* data, int s_merge) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const uint64_t base = (uint64_t)blockIdx.x << LT;
  T* g = data + base;
  const uint32_t t = threadIdx.x;
  T v[16];
  // window LT-4: thread t takes elements t + r * 2^(LT-4): coalesced loads
#pragma unroll
  for (int r = 0; r < 16; r++) v[r] = g[win_idx<LT - 4>(t, r)];
  if (((base >> s_merge) & 1) == 0)
    merge_chunks<LT, LT - 1, LT - 4, true>(sm, v, g);
  else
    merge_chunks<LT, LT - 1, LT - 4, false>(sm, v, g);
}

template <int NB, bool ASC>
__device__ __forceinline__ void global_steps(ulonglong2* v) {
  constexpr int E = 1 << NB;
#pragma unroll
  for (int b = NB - 1; b >= 0; b--) {
#pragma unroll
    for (int r = 0; r < E; r++) {
      if (r & (1 << b)) continue;
      uint64_t a0 = v[r].x, a1 = v[r].y, c0 = v[r | (1 << b)].x, c1 = v[r | (1 << b)].y;
      cxd<ASC>(a0, c0);
      cxd<ASC>(a1, c1);
      v[r] = make_ulonglong2(a0, a1);
      v[r | (1 << b)] = make_ulonglong2(c0, c1);
    }
  }
}

// Steps b = b_hi .. b_hi-NB+1 (all >= the tile bits) of stage s, one HBM pass.
// Thread t owns the pair of adjacent low positions (2u, 2u+1) and the 2^NB
// positions that differ in the stride bits.
template <int NB>
__global__ void __launch_bounds__(256, 2) k_sort_global_u64(uint64_t* data, uint64_t n, int s,
                                                         int b_hi) {
  constexpr int E = 1 << NB;
  const int w_lo = b_hi - NB + 1;
  const uint64_t nthreads = n / (2 * E);
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nthreads;
       t += (uint64_t)gridDim.x * blockDim.x) {
    // t indexes element pairs: low part (w_lo - 1 bits) and high part
    const uint64_t low = (t << 1) & ((1ull << w_lo) - 1);
    const uint64_t high = (t << 1) >> w_lo;
    const uint64_t base = (high << (w_lo + NB)) | low;
    ulonglong2 v[E];
#pragma unroll
    for (int r = 0; r < E; r++)
      v[r] = *reinterpret_cast<const ulonglong2*>(data + (base | ((uint64_t)r << w_lo)));
    // bit s is above every stride bit: one direction per thread
    if (((base >> s) & 1) == 0)
      global_steps<NB, true>(v);
    else
      global_steps<NB, false>(v);
#pragma unroll
    for (int r = 0; r < E; r++)
      *reinterpret_cast<ulonglong2*>(data + (base | ((uint64_t)r << w_lo))) = v[r];
  }
}

template <int LT, typename T = uint64_t>
static size_t tile_smem() {
  return (size_t)((1u << LT) + (1u << LT) / 16) * sizeof(T);
}

template <int LT>
static cudaError_t sort_u64_lt(uint64_t* tags, uint64_t n, cudaStream_t st,
                               int cls_global = P_SORT_GLOBAL, int cls_tile = P_SORT_TILE) {
  const size_t smem = tile_smem<LT>();
  {
    cudaError_t e = raise_smem_limit((const void*)k_sort_tile_full<LT, uint64_t>, smem);
    if (e == cudaSuccess) e = raise_smem_limit((const void*)k_sort_tile_merge<LT, uint64_t>, smem);
    if (e != cudaSuccess) return e;
  }
  const uint64_t tiles = n >> LT;
  const int nt = 1 << (LT - 4);
  {
    ProfSpan ps(cls_tile, st);
    k_sort_tile_full<LT, uint64_t><<<(unsigned)tiles, nt, smem, st>>>(tags);
    count_launch();
  }
  int logn = 0;
  while ((1ull << logn) < n) logn++;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int s = LT + 1; s <= logn; s++) {
    for (int hi = s - 1; hi >= LT; hi -= 4) {
      const int nb = hi - LT + 1 < 4 ? hi - LT + 1 : 4;
      const uint64_t threads = n / (2ull << nb);
      const uint64_t blocks = (threads + 255) / 256;
      const uint64_t cap = (uint64_t)sms * 16;
      const unsigned g = (unsigned)(blocks < cap ? blocks : cap);
      ProfSpan ps(cls_global, st);
      count_launch();
      switch (nb) {
        case 1: k_sort_global_u64<1><<<g, 256, 0, st>>>(tags, n, s, hi); break;
        case 2: k_sort_global_u64<2><<<g, 256, 0, st>>>(tags, n, s, hi); break;
        case 3: k_sort_global_u64<3><<<g, 256, 0, st>>>(tags, n, s, hi); break;
        default: k_sort_global_u64<4><<<g, 256, 0, st>>>(tags, n, s, hi); break;
      }
    }
    ProfSpan ps(cls_tile, st);
    k_sort_tile_merge<LT, uint64_t><<<(unsigned)tiles, nt, smem, st>>>(tags, s);
    count_launch();
  }
  return cudaGetLastError();
}

// n must be a power of two and at least 2^log_tile.
cudaError_t sort_tags_u64(uint64_t* tags, uint64_t n, int log_tile, cudaStream_t st,
                          int cls_global, int cls_tile) {
  if (n & (n - 1)) return cudaErrorInvalidValue;
  if (log_tile == 13 && n >= (1ull << 13)) return sort_u64_lt<13>(tags, n, st, cls_global, cls_tile);
  if (log_tile == 12 && n >= (1ull << 12)) return sort_u64_lt<12>(tags, n, st, cls_global, cls_tile);
  if (log_tile == 9 && n >= (1ull << 9)) return sort_u64_lt<9>(tags, n, st, cls_global, cls_tile);
  return cudaErrorInvalidValue;
}

// batch grouping keys packed in 32 bits: one tile of n = 512 or 4096 keys
cudaError_t sort_batch_keys32(uint32_t* keys, uint32_t n, cudaStream_t st) {
  if (n == 512) {
    k_sort_tile_full<9, uint32_t><<<1, 32, tile_smem<9, uint32_t>(), st>>>(keys);
  } else if (n == 4096) {
    k_sort_tile_full<12, uint32_t><<<1, 256, tile_smem<12, uint32_t>(), st>>>(keys);
  } else {
    return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

// batch grouping keys, n a power of two in [512, 65536]
cudaError_t sort_batch_keys(uint64_t* keys, uint32_t n, cudaStream_t st) {
  if (n == 512) return sort_u64_lt<9>(keys, n, st);
  if (n < 4096 || n > 65536 || (n & (n - 1))) return cudaErrorInvalidValue;
  return sort_u64_lt<12>(keys, n, st);
}

}  // namespace bdev
