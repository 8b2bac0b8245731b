// rr_build.cu -- scene ingest and LBVH build on the GPU.
//
// Steps (all stream ordered, no host round trip):
//   a1 ingest    validate indices, per-triangle centroid, scene centroid bounds
//   a2 Morton    30-bit codes of the centroids normalised to the bounds
//   a3 sort      stable LSD radix sort of (code, triangle id), 4 passes of 8 bits
//   a4 Karras    internal-node ranges and splits from the sorted codes
//                (Karras, "Maximizing parallelism in the construction of BVHs,
//                octrees, and k-d trees", HPG 2012), equal codes ordered by index
//   a5 refit     bottom-up child boxes, the second child to arrive merges
//   a5b SAH top  (RR_BVH_SAH_TOP) the part of the tree above its subtrees of
//                at most kClusterMax leaves rebuilt top down by binned SAH
//                over those subtrees, in the node slots it frees
// plus the per-material lobe table of Eq. 5 used by the beam window (Eq. 4).
//
// The hierarchy is a binary BVH with one triangle per leaf.  Internal node i
// is stored as four float4 (Aila & Laine, HPG 2009 layout):
//   n0 = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)   n1 = same for child 1
//   n2 = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)   n3 = (child0, child1, 0, 0)
// with a child reference i for internal node i and j | 0x80000000 for leaf j.
// Leaves are the triangles in sorted order: tri[3j..3j+2] = v0, v1, v2 with
// v0.w = original triangle id, v1.w = material id (bit patterns).
#include <algorithm>
#include <cstring>
#include <cuda/atomic>
#include <cuda_runtime.h>

#include "rr_host.h"

namespace rr {

constexpr int kSortBlock = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortBlock * kSortItems;

// order-preserving map of floats to unsigned for atomic min / max
__device__ __forceinline__ uint32_t enc_f(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float dec_f(uint32_t e) {
  return __uint_as_float((e & 0x80000000u) ? (e & 0x7FFFFFFFu) : ~e);
}

// device-scope acquire loads and release stores of the bounded producer /
// consumer waits in the SAH top and the wide collapse
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// a1: validation, centroids and centroid bounds
// misc[0..2] = encoded min xyz, misc[3..5] = encoded max xyz, misc[6] = error
__global__ void k_ingest(const float* __restrict__ vtx, const uint32_t* __restrict__ idx,
                         const uint16_t* __restrict__ mat_id, uint32_t nv, uint32_t nt, uint32_t nm,
                         float4* __restrict__ centroid, uint32_t* __restrict__ misc) {
  __shared__ float s_lo[3][32], s_hi[3][32];
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  if (i < nt) {
    uint32_t err = 0;
    const uint32_t a = idx[3 * i], b = idx[3 * i + 1], c = idx[3 * i + 2];
    if (a >= nv || b >= nv || c >= nv) err |= 1u;
    if (mat_id[i] >= nm) err |= 2u;
    float cen[3] = {0.f, 0.f, 0.f};
    if (!(err & 1u)) {
      for (int k = 0; k < 3; ++k) {
        const float x0 = vtx[3 * a + k], x1 = vtx[3 * b + k], x2 = vtx[3 * c + k];
        if (!isfinite(x0) || !isfinite(x1) || !isfinite(x2)) err |= kErrBadVertex;
        cen[k] = (x0 + x1 + x2) / 3.0f;
      }
    }
    if (err) {
      atomicOr(&misc[6], err);
    } else {
      for (int k = 0; k < 3; ++k) lo[k] = hi[k] = cen[k];
    }
    centroid[i] = make_float4(cen[0], cen[1], cen[2], 0.f);
  }
  // warp then block reduction of the bounds
  for (int k = 0; k < 3; ++k) {
    for (int off = 16; off > 0; off >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xFFFFFFFFu, lo[k], off));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xFFFFFFFFu, hi[k], off));
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0)
    for (int k = 0; k < 3; ++k) {
      s_lo[k][warp] = lo[k];
      s_hi[k][warp] = hi[k];
    }
  __syncthreads();
  if (warp == 0) {
    for (int k = 0; k < 3; ++k) {
      float l = lane < nw ? s_lo[k][lane] : INFINITY, h = lane < nw ? s_hi[k][lane] : -INFINITY;
      for (int off = 16; off > 0; off >>= 1) {
        l = fminf(l, __shfl_xor_sync(0xFFFFFFFFu, l, off));
        h = fmaxf(h, __shfl_xor_sync(0xFFFFFFFFu, h, off));
      }
      if (lane == 0 && l <= h) {
        atomicMin(&misc[k], enc_f(l));
        atomicMax(&misc[3 + k], enc_f(h));
      }
    }
  }
}

// spread the low 10 bits of v so that bit i lands on bit 3i
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

// a2: code = x9 y9 z9 x8 y8 z8 ... x0 y0 z0 of the quantised centroid
// also counts the first sort pass's digits per tile (hist0, zeroed before)
__global__ void k_morton(const float4* __restrict__ centroid, const uint32_t* __restrict__ misc, uint32_t nt,
                         uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, uint32_t tiles,
                         uint32_t* __restrict__ hist0) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nt) return;
  const float4 c = centroid[i];
  const float cc[3] = {c.x, c.y, c.z};
  uint32_t q[3];
  for (int k = 0; k < 3; ++k) {
    const float lo = dec_f(misc[k]), hi = dec_f(misc[3 + k]);
    const float ext = hi - lo;
    const float x = ext > 0.0f ? (cc[k] - lo) / ext : 0.0f;
    q[k] = (uint32_t)fminf(floorf(x * 1024.0f), 1023.0f);
  }
  const uint32_t key = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
  keys[i] = key;
  vals[i] = i;
  atomicAdd(&hist0[(key & 255u) * tiles + i / kSortTile], 1u);
}

// ---------------------------------------------------------------------------
// a3: LSD radix sort, 8-bit digits, stable.  Each pass's digit counts per
// tile of its input (digit major: hist[d * tiles + t]) are counted while that
// input is written -- by k_morton for the first pass, by the previous pass's
// scatter (a key's tile in the next pass is its output position / tile)
// for the others -- then scanned by k_scan_single into the scatter offsets.

// exclusive scan of n counters (n a multiple of 4, 16-byte aligned) with one
// block.  Up to 8 uint4 per thread: each thread loads its contiguous run at
// once (one round trip), one block scan of the run sums.  More: chunks of
// blockDim x 4 counters, one coalesced uint4 per thread, carried from chunk
// to chunk.
__global__ void k_scan_single(uint32_t* __restrict__ data, uint32_t n) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  const uint32_t t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  uint4* d4 = reinterpret_cast<uint4*>(data);
  const uint32_t n4 = n / 4u;
  const uint32_t per = (n4 + blockDim.x - 1) / blockDim.x;
  if (per <= 8u) {
    const uint32_t b0 = t * per;
    uint4 v[8];
    uint32_t sum = 0;
#pragma unroll
    for (uint32_t k = 0; k < 8u; ++k) {
      v[k] = make_uint4(0u, 0u, 0u, 0u);
      if (k < per && b0 + k < n4) v[k] = d4[b0 + k];
    }
#pragma unroll
    for (uint32_t k = 0; k < 8u; ++k) sum += v[k].x + v[k].y + v[k].z + v[k].w;
    uint32_t x = sum;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = lane < nw ? s_warp[lane] : 0u;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, off);
        if (lane >= off) w += y;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    uint32_t run = x - sum + (warp > 0 ? s_warp[warp - 1] : 0u);
#pragma unroll
    for (uint32_t k = 0; k < 8u; ++k) {
      if (k < per && b0 + k < n4) {
        uint4 o;
        o.x = run;
        run += v[k].x;
        o.y = run;
        run += v[k].y;
        o.z = run;
        run += v[k].z;
        o.w = run;
        run += v[k].w;
        d4[b0 + k] = o;
      }
    }
    return;
  }
  if (t == 0) s_carry = 0u;
  __syncthreads();
  for (uint32_t base = 0; base < n4; base += blockDim.x) {
    const uint32_t i = base + t;
    uint4 v = i < n4 ? d4[i] : make_uint4(0u, 0u, 0u, 0u);
    const uint32_t sum = v.x + v.y + v.z + v.w;
    uint32_t x = sum;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = lane < nw ? s_warp[lane] : 0u;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, off);
        if (lane >= off) w += y;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t carry = s_carry;
    uint32_t run = carry + x - sum + (warp > 0 ? s_warp[warp - 1] : 0u);
    if (i < n4) {
      uint4 o;
      o.x = run;
      run += v.x;
      o.y = run;
      run += v.y;
      o.z = run;
      run += v.z;
      o.w = run;
      d4[i] = o;
    }
    __syncthreads();
    if (t == 0) s_carry = carry + s_warp[nw - 1];
    __syncthreads();
  }
}

// Exclusive scan of counter arrays too long for one block to scan in one
// round trip (the 5M-triangle sort has 625k counters per pass): the counters
// are split into tiles of kScanTile, 16 consecutive counters per thread;
// k_scan_tiles_up writes each tile's sum, k_scan_single scans the sums,
// k_scan_tiles_down scans each tile from its offset.  Three launches of about
// one block per SM instead of one block walking the whole array.
constexpr int kScanBlock = 256;
constexpr uint32_t kScanTile = kScanBlock * 16u;
// counters k_scan_single scans in one round trip (8 uint4 per thread, 1024 threads)
constexpr uint32_t kScanSingleMax = 8u * 4u * 1024u;

__host__ __device__ constexpr uint32_t scan_tiles(size_t n) { return (uint32_t)((n + kScanTile - 1) / kScanTile); }
// words of tile sums (a multiple of 4, as k_scan_single wants)
__host__ __device__ constexpr uint32_t scan_tile_words(size_t n) { return (scan_tiles(n) + 3u) & ~3u; }

// block-wide sum of one value per thread (every thread gets the sum)
__device__ __forceinline__ uint32_t block_sum(uint32_t x, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, off);
  if (lane == 0) s_warp[warp] = x;
  __syncthreads();
  uint32_t t = 0;
  for (int w = 0; w < kScanBlock / 32; ++w) t += s_warp[w];
  return t;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_tiles_up(const uint32_t* __restrict__ data, uint32_t n4,
                                                              uint32_t* __restrict__ tsum, uint32_t tsum_words) {
  __shared__ uint32_t s_warp[kScanBlock / 32];
  const uint4* d4 = reinterpret_cast<const uint4*>(data);
  const uint32_t b4 = blockIdx.x * (kScanTile / 4u) + threadIdx.x * 4u;
  uint32_t sum = 0;
#pragma unroll
  for (uint32_t k = 0; k < 4u; ++k)
    if (b4 + k < n4) {
      const uint4 v = d4[b4 + k];
      sum += v.x + v.y + v.z + v.w;
    }
  const uint32_t t = block_sum(sum, s_warp);
  if (threadIdx.x == 0) tsum[blockIdx.x] = t;
  // the padding words after the last tile's sum
  if (blockIdx.x == 0 && gridDim.x + threadIdx.x < tsum_words) tsum[gridDim.x + threadIdx.x] = 0u;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_tiles_down(uint32_t* __restrict__ data, uint32_t n4,
                                                                const uint32_t* __restrict__ tsum) {
  __shared__ uint32_t s_warp[kScanBlock / 32];
  uint4* d4 = reinterpret_cast<uint4*>(data);
  const uint32_t b4 = blockIdx.x * (kScanTile / 4u) + threadIdx.x * 4u;
  uint4 v[4];
  uint32_t sum = 0;
#pragma unroll
  for (uint32_t k = 0; k < 4u; ++k) {
    v[k] = b4 + k < n4 ? d4[b4 + k] : make_uint4(0u, 0u, 0u, 0u);
    sum += v[k].x + v[k].y + v[k].z + v[k].w;
  }
  // exclusive prefix of the per-thread sums within the tile
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = sum;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  uint32_t run = tsum[blockIdx.x] + x - sum;
  for (int w = 0; w < warp; ++w) run += s_warp[w];
#pragma unroll
  for (uint32_t k = 0; k < 4u; ++k) {
    if (b4 + k < n4) {
      uint4 o;
      o.x = run;
      run += v[k].x;
      o.y = run;
      run += v[k].y;
      o.z = run;
      run += v[k].z;
      o.w = run;
      run += v[k].w;
      d4[b4 + k] = o;
    }
  }
}

// stable scatter: keys of a tile are ranked in index order (round, warp, lane).
// The tile's keys and values are loaded up front (one round trip instead of
// one per round); lanes with the same digit are found with 8 ballots.  With
// hist_next, each key is also counted for the next pass (digit shift + 8).
__global__ void k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, uint32_t n, int shift,
                                uint32_t tiles, const uint32_t* __restrict__ offs, uint32_t* __restrict__ hist_next) {
  __shared__ uint32_t s_base[256];
  __shared__ uint32_t s_warp[kSortBlock / 32][256];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  s_base[t] = offs[t * tiles + blockIdx.x];
  const uint32_t base = blockIdx.x * kSortTile;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t keys[kSortItems], vals[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const uint32_t i = base + r * kSortBlock + t;
    keys[r] = i < n ? kin[i] : 0u;
    vals[r] = i < n ? vin[i] : 0u;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    for (int w = 0; w < kSortBlock / 32; ++w) s_warp[w][t] = 0;
    __syncthreads();
    const uint32_t i = base + r * kSortBlock + t;
    const bool valid = i < n;
    const uint32_t key = keys[r];
    const uint32_t digit = (key >> shift) & 255u;
    // lanes holding the same digit: agree on all 8 bits; invalid lanes
    // (only in the last tile, always the highest lanes) match nobody
    uint32_t peers = __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const uint32_t ones = __ballot_sync(0xFFFFFFFFu, (digit >> b) & 1u);
      peers &= ((digit >> b) & 1u) ? ones : ~ones;
    }
    const uint32_t rank = __popc(peers & lt_mask);
    if (valid && rank == 0) s_warp[warp][digit] = __popc(peers);
    __syncthreads();
    uint32_t acc = 0;
    for (int w = 0; w < kSortBlock / 32; ++w) {
      const uint32_t c = s_warp[w][t];
      s_warp[w][t] = acc;
      acc += c;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = s_base[digit] + s_warp[warp][digit] + rank;
      kout[pos] = key;
      vout[pos] = vals[r];
      if (hist_next) atomicAdd(&hist_next[((key >> (shift + 8)) & 255u) * tiles + pos / kSortTile], 1u);
    }
    __syncthreads();
    s_base[t] += acc;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// sorted leaves: triangle data in leaf order, leaf boxes
__global__ void k_gather(const float* __restrict__ vtx, const uint32_t* __restrict__ idx,
                         const uint16_t* __restrict__ mat_id, const uint32_t* __restrict__ perm, uint32_t nv,
                         uint32_t nt,
                         float4* __restrict__ tri, float* __restrict__ nbox) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nt) return;
  const uint32_t t = perm[j];
  float3 v[3];
  for (int c = 0; c < 3; ++c) {
    const uint32_t vi = idx[3 * t + c];
    // an invalid index was flagged by the ingest step; never read past the vertices
    v[c] = vi < nv ? make_float3(vtx[3 * vi], vtx[3 * vi + 1], vtx[3 * vi + 2]) : make_float3(0.f, 0.f, 0.f);
  }
  {   // the unit normal (and the material) after the three copies
    const float3 nr = normalize(cross(v[1] - v[0], v[2] - v[0]));
    tri[(size_t)kTriCopies * 3 * nt + j] = make_float4(nr.x, nr.y, nr.z, __uint_as_float((uint32_t)mat_id[t]));
  }
  const float w[3] = {__uint_as_float(t), __uint_as_float((uint32_t)mat_id[t]), 0.0f};
#pragma unroll
  for (uint32_t r = 0; r < (uint32_t)kTriCopies; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float3 u = tri_rotate(v[c], r);
      tri[(size_t)r * 3 * nt + 3 * (size_t)j + c] = make_float4(u.x, u.y, u.z, w[c]);
    }
  float* b = nbox + 6 * (size_t)(nt - 1 + j);
  b[0] = fminf(fminf(v[0].x, v[1].x), v[2].x);
  b[1] = fminf(fminf(v[0].y, v[1].y), v[2].y);
  b[2] = fminf(fminf(v[0].z, v[1].z), v[2].z);
  b[3] = fmaxf(fmaxf(v[0].x, v[1].x), v[2].x);
  b[4] = fmaxf(fmaxf(v[0].y, v[1].y), v[2].y);
  b[5] = fmaxf(fmaxf(v[0].z, v[1].z), v[2].z);
}

// common-prefix length of sorted keys i and j; equal keys compare their indices
__device__ __forceinline__ int delta(const uint32_t* __restrict__ k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  const uint32_t a = k[i], b = k[j];
  if (a == b) return 32 + __clz((uint32_t)i ^ (uint32_t)j);
  return __clz(a ^ b);
}

// a4: internal node i covers a key range that starts or ends at i; its split
// is the highest position where the common prefix shrinks
__global__ void k_karras(const uint32_t* __restrict__ keys, int n, uint32_t* __restrict__ child,
                         uint32_t* __restrict__ parent, uint32_t* __restrict__ visit, uint2* __restrict__ range) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  const int dmin = delta(keys, n, i, i - d);
  int lmax = 2;
  while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
  const int j = i + l * d;
  const int dnode = delta(keys, n, i, j);
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  const int gamma = i + s * d + min(d, 0);
  const int lo = min(i, j), hi = max(i, j);
  const uint32_t left = (lo == gamma) ? ((uint32_t)gamma | kLeafBit) : (uint32_t)gamma;
  const uint32_t right = (hi == gamma + 1) ? ((uint32_t)(gamma + 1) | kLeafBit) : (uint32_t)(gamma + 1);
  child[2 * i] = left;
  child[2 * i + 1] = right;
  range[i] = make_uint2((uint32_t)lo, (uint32_t)hi);
  parent[(left & kLeafBit) ? (n - 1 + (left & ~kLeafBit)) : left] = (uint32_t)i;
  parent[(right & kLeafBit) ? (n - 1 + (right & ~kLeafBit)) : right] = (uint32_t)i;
  visit[i] = 0;
  if (i == 0) parent[0] = kNone;
}

__device__ __forceinline__ uint32_t node_slot(uint32_t c, uint32_t n) {
  return (c & kLeafBit) ? (n - 1 + (c & ~kLeafBit)) : c;
}

// Members of a wide node's cut: a triangle (kLeafBit | leaf), a small binary
// subtree of 2..kGroupMax triangles held in one leaf slot (kGroupBit |
// count << kGroupShift | binary node), or a binary node that becomes a wide
// node of its own; kNone for an empty slot.
constexpr uint32_t kGroupBit = 1u << 30;
constexpr uint32_t kGroupShift = 28;
constexpr uint32_t kGroupNodeMask = (1u << kGroupShift) - 1u;
// At most two triangles per group: on the 200k- and 5M-triangle scenes that
// removes 45 % of the wide nodes for about 1 % more query time; groups of
// three remove 52-57 % and cost 2-4 % (a leaf slot's triangles are all
// tested once its box is hit).  The count field has room for three.
constexpr uint32_t kGroupMax = 2;

__device__ __forceinline__ bool member_is_group(uint32_t m) { return m != kNone && !(m & kLeafBit) && (m & kGroupBit); }
__device__ __forceinline__ bool member_is_inner(uint32_t m) { return m != kNone && !(m & (kLeafBit | kGroupBit)); }
// triangles a leaf slot holds (0: an inner member or an empty slot)
__device__ __forceinline__ uint32_t member_tris(uint32_t m) {
  if (m == kNone) return 0u;
  if (m & kLeafBit) return 1u;
  return (m & kGroupBit) ? (m >> kGroupShift) & 3u : 0u;
}
// the member's slot in the node boxes (a group: its binary node)
__device__ __forceinline__ uint32_t member_box(uint32_t m, uint32_t n) {
  return member_is_group(m) ? (m & kGroupNodeMask) : node_slot(m, n);
}

// a binary child reference classified as a member: a subtree of at most
// kGroupMax triangles (at most kGroupMax - 1 internal nodes) becomes a group
__device__ __forceinline__ uint32_t classify_member(uint32_t c, const uint32_t* __restrict__ child) {
  if ((c & kLeafBit) || kGroupMax < 2) return c;
  uint32_t stack[kGroupMax], sp = 0, tris = 0, inner = 0;
  stack[sp++] = c;
  while (sp) {
    const uint32_t x = stack[--sp];
    if (x & kLeafBit) {
      ++tris;
      continue;
    }
    if (++inner > kGroupMax - 1 || sp + 2 > kGroupMax) return c;
    stack[sp++] = __ldg(&child[2 * x]);
    stack[sp++] = __ldg(&child[2 * x + 1]);
  }
  return (tris <= kGroupMax && c < (1u << kGroupShift)) ? (kGroupBit | (tris << kGroupShift) | c) : c;
}

// a5: each leaf walks to the root; at every internal node the first arrival
// stops and the second merges both child boxes (they are final by then).
// The walker carries the box of the child it comes from, so it reads only
// the sibling's; the node's children and parent are read alongside the
// arrival atomic (they do not depend on it).  A node whose leaf range lies
// inside the block's own leaves (so does its index: a Karras node is one end
// of its range) is merged through shared memory -- arrival counter and child
// boxes -- so the bottom levels of every walk cost no L2 round trips; the
// others through the global counters and nbox.
constexpr int kRefitBlock = 256;
__global__ void __launch_bounds__(kRefitBlock) k_refit(uint32_t n, const uint32_t* __restrict__ child,
                                                       const uint32_t* __restrict__ parent,
                                                       const uint2* __restrict__ range, uint32_t* __restrict__ visit,
                                                       float* __restrict__ nbox, float4* __restrict__ nodes) {
  __shared__ float s_box[2][kRefitBlock][6];   // [0] the block's leaves, [1] its local internal nodes
  __shared__ uint32_t s_visit[kRefitBlock];
  const uint32_t base = blockIdx.x * kRefitBlock, end = min(base + kRefitBlock, n);
  const uint32_t j = base + threadIdx.x;
  s_visit[threadIdx.x] = 0u;
  float own[6];
  if (j < n)
    for (int k = 0; k < 6; ++k) {
      own[k] = __ldcg(nbox + 6 * (size_t)(n - 1 + j) + k);
      s_box[0][threadIdx.x][k] = own[k];
    }
  __syncthreads();
  if (j >= n) return;
  uint32_t cur = j | kLeafBit;
  uint32_t p = __ldg(&parent[n - 1 + j]);
  while (p != kNone) {
    const uint32_t c0 = __ldg(&child[2 * p]), c1 = __ldg(&child[2 * p + 1]);
    const uint32_t pp = __ldg(&parent[p]);
    const uint2 rg = __ldg(&range[p]);
    const bool local = rg.x >= base && rg.y < end;
    const bool first_is_own = c0 == cur;
    const uint32_t sib = first_is_own ? c1 : c0;
    float sb[6];
    if (local) {
      // fence - atomic - fence: the sibling's box, written before its
      // walker arrived, is visible to the second arrival
      __threadfence_block();
      if (atomicAdd(&s_visit[p - base], 1u) == 0u) return;
      __threadfence_block();
      const float* q = (sib & kLeafBit) ? s_box[0][(sib & ~kLeafBit) - base] : s_box[1][sib - base];
      for (int k = 0; k < 6; ++k) sb[k] = q[k];
    } else {
      // acquire-release: the second arrival sees the first one's box
      cuda::atomic_ref<uint32_t, cuda::thread_scope_device> cnt(visit[p]);
      if (cnt.fetch_add(1u, cuda::memory_order_acq_rel) == 0u) return;
      const float* q = nbox + 6 * (size_t)node_slot(sib, n);
      for (int k = 0; k < 6; ++k) sb[k] = __ldcg(q + k);
    }
    float b0[6], b1[6];
    for (int k = 0; k < 6; ++k) {
      b0[k] = first_is_own ? own[k] : sb[k];
      b1[k] = first_is_own ? sb[k] : own[k];
    }
    float4* nd = nodes + 4 * (size_t)p;
    nd[0] = make_float4(b0[0], b0[3], b0[1], b0[4]);
    nd[1] = make_float4(b1[0], b1[3], b1[1], b1[4]);
    nd[2] = make_float4(b0[2], b0[5], b1[2], b1[5]);
    nd[3] = make_float4(__uint_as_float(c0), __uint_as_float(c1), 0.f, 0.f);
    float* bp = nbox + 6 * (size_t)p;
    for (int k = 0; k < 3; ++k) {
      own[k] = fminf(b0[k], b1[k]);
      own[3 + k] = fmaxf(b0[3 + k], b1[3 + k]);
      __stcg(bp + k, own[k]);
      __stcg(bp + 3 + k, own[3 + k]);
    }
    if (local)
      for (int k = 0; k < 6; ++k) s_box[1][p - base][k] = own[k];
    cur = p;
    p = pp;
  }
}

// depth of every leaf (number of internal ancestors), maximum into misc[7]
__global__ void k_depth(uint32_t n, const uint32_t* __restrict__ parent, uint32_t* __restrict__ misc) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  uint32_t d = 0, p = parent[n - 1 + j];
  while (p != kNone && d < 4096u) {
    ++d;
    p = parent[p];
  }
  atomicMax(&misc[7], d);
}

// ---------------------------------------------------------------------------
// a5b: SAH top (HLBVH: Pantaleoni and Luebke, HPG 2010; Garanzha, Pantaleoni
// and McAllister, HPG 2011).  The clusters are the LBVH's maximal subtrees of
// at most kClusterMax leaves, in leaf order; the C - 1 internal nodes above
// them are rebuilt top down by binned SAH over the clusters (box = union of
// the subtree, weight = its leaves), reusing exactly their node slots with
// the root kept at 0.  A task over clusters [b, e) at depth d:
//   centroid c = 0.5 (lo + hi); bounds cmin, cmax; per axis with
//   ext = cmax - cmin > 0: scale = kTopBins / ext, bin
//   q = min(kTopBins - 1, trunc((c - cmin) scale)), each step rounded to float;
//   a split after bin q with both sides non-empty costs
//   area(L) weight(L) + area(R) weight(R) (float, area = dx dy + dy dz + dz dx);
//   the lowest cost wins, ties to the lower axis, then the lower q; without a
//   split, or at depth >= kTopMedianDepth, the first n / 2 clusters go left.
//   The partition keeps the order on each side; a side of one cluster is that
//   cluster's subtree, otherwise a new task at d + 1.
// Every operation is exactly rounded, so a host restatement of these rules
// builds the same tree.  Tasks of more than kTopSmall clusters are worked by
// whole blocks (k_top_sah), smaller ones by one warp each (k_top_small).
constexpr uint32_t kClusterMax = 32;
constexpr int kTopBins = 32;
constexpr uint32_t kTopMedianDepth = 32;
constexpr int kTopBlock = 512;
constexpr uint32_t kTopSmall = 32;            // a warp task: at most one cluster per lane
constexpr int kClTile = 2048;                 // compaction: 256 threads x 8 leaves
constexpr uint32_t kTopSpinLimit = 1u << 22;  // x <= 256 ns naps: about a second
// counters of the SAH top
constexpr int kCtrHead = 0;       // next block task to take
constexpr int kCtrSlots = 1;      // node slots handed out after the root
constexpr int kCtrMarked = 2;     // top slots found after the root (k_top_mark)
constexpr int kCtrClusters = 3;   // C
constexpr int kCtrTasks = 4;      // block tasks created
constexpr int kCtrPending = 5;    // block tasks created and not finished
constexpr int kCtrSmall = 6;      // warp tasks created
constexpr int kCtrSmallHead = 7;  // next warp task to take

// top part and clusters: internal node i is a top node when it has more than
// kClusterMax leaves; a child of a top node with at most kClusterMax leaves
// is a cluster root, recorded at its first leaf
__global__ void k_top_mark(uint32_t n, const uint32_t* __restrict__ child, const uint2* __restrict__ range,
                           uint32_t* __restrict__ cl_at, uint32_t* __restrict__ slot, uint32_t* __restrict__ ctr,
                           uint32_t* __restrict__ cb) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i + 1 >= n) return;
  const uint2 r = range[i];
  if (r.y - r.x + 1u <= kClusterMax) return;
  if (i == 0) {
    slot[0] = 0u;
    for (int k = 0; k < 3; ++k) {   // the root task's centroid bounds, filled by k_top_compact
      cb[k] = 0xFF800000u;          // enc_f(+inf)
      cb[3 + k] = 0x007FFFFFu;      // enc_f(-inf)
    }
  } else {
    slot[1u + atomicAdd(&ctr[kCtrMarked], 1u)] = i;
  }
  for (int k = 0; k < 2; ++k) {
    const uint32_t c = child[2 * i + k];
    uint32_t first, size;
    if (c & kLeafBit) {
      first = c & ~kLeafBit;
      size = 1u;
    } else {
      const uint2 rc = range[c];
      first = rc.x;
      size = rc.y - rc.x + 1u;
    }
    if (size <= kClusterMax) cl_at[first] = c;
  }
}

// clusters of each block of kClTile leaves
__global__ void __launch_bounds__(256) k_top_count(uint32_t n, const uint32_t* __restrict__ cl_at,
                                                   uint32_t* __restrict__ bsum) {
  __shared__ uint32_t s_w[8];
  const uint32_t base = blockIdx.x * kClTile + threadIdx.x * 8u;
  uint32_t c = 0;
  for (uint32_t k = 0; k < 8; ++k)
    if (base + k < n && cl_at[base + k] != kNone) ++c;
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, off);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    bsum[blockIdx.x] = t;
  }
}

// clusters in leaf order (bsum holds the exclusive block offsets): their
// records, and the root task over all of them
__global__ void __launch_bounds__(256) k_top_compact(uint32_t n, const uint32_t* __restrict__ cl_at,
                                                     const uint32_t* __restrict__ bsum, const uint2* __restrict__ range,
                                                     const float* __restrict__ nbox, float4* __restrict__ rec,
                                                     uint4* __restrict__ task,
                                                     uint32_t* __restrict__ ready, uint4* __restrict__ small,
                                                     uint32_t* __restrict__ ctr, uint32_t* __restrict__ cb) {
  __shared__ uint32_t s_w[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t base = blockIdx.x * kClTile + threadIdx.x * 8u;
  uint32_t c = 0;
  for (uint32_t k = 0; k < 8; ++k)
    if (base + k < n && cl_at[base + k] != kNone) ++c;
  uint32_t x = c;   // inclusive scan over the warp
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  uint32_t pos = bsum[blockIdx.x] + x - c;
  for (int w = 0; w < warp; ++w) pos += s_w[w];
  float cmn[3] = {INFINITY, INFINITY, INFINITY}, cmx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (uint32_t k = 0; k < 8; ++k) {
    const uint32_t j = base + k;
    if (j >= n) break;
    const uint32_t ref = cl_at[j];
    if (ref != kNone) {
      const uint32_t slot = (ref & kLeafBit) ? (n - 1 + (ref & ~kLeafBit)) : ref;
      const float* b = nbox + 6 * (size_t)slot;
      uint32_t weight = 1u;
      if (!(ref & kLeafBit)) {
        const uint2 r = range[ref];
        weight = r.y - r.x + 1u;
      }
      rec[2 * (size_t)pos] = make_float4(b[0], b[1], b[2], __uint_as_float(weight));
      rec[2 * (size_t)pos + 1] = make_float4(b[3], b[4], b[5], __uint_as_float(ref));
      for (int q = 0; q < 3; ++q) {
        const float c = __fmul_rn(0.5f, __fadd_rn(b[q], b[3 + q]));
        cmn[q] = fminf(cmn[q], c);
        cmx[q] = fmaxf(cmx[q], c);
      }
      ++pos;
    }
    if (j == n - 1) {   // the last leaf: pos is now the number of clusters
      ctr[kCtrClusters] = pos;
      if (pos > kTopSmall) {
        task[0] = make_uint4(0u, pos, 0u, 0u);
        ready[0] = 1u;
        ctr[kCtrTasks] = 1u;
        ctr[kCtrPending] = 1u;
      } else {
        small[0] = make_uint4(0u, pos, 0u, 0u);
        ctr[kCtrSmall] = 1u;
      }
    }
  }
  for (int q = 0; q < 3; ++q)
    for (int off = 16; off > 0; off >>= 1) {
      cmn[q] = fminf(cmn[q], __shfl_xor_sync(0xFFFFFFFFu, cmn[q], off));
      cmx[q] = fmaxf(cmx[q], __shfl_xor_sync(0xFFFFFFFFu, cmx[q], off));
    }
  if (lane == 0 && cmn[0] <= cmx[0])
    for (int q = 0; q < 3; ++q) {
      atomicMin(&cb[q], enc_f(cmn[q]));
      atomicMax(&cb[3 + q], enc_f(cmx[q]));
    }
}

struct TopArgs {
  float4* rec[2];         // [C][2] cluster records, ping-pong between a task and its children
  const uint32_t* slot;   // [C - 1] node slots of the top part, root first
  uint4* task;            // [C - 1] block tasks (more than kTopSmall clusters)
  uint32_t* ready;        // [C - 1] block task published
  uint4* small;           // [C - 1] warp tasks (2 to kTopSmall clusters)
  uint32_t* ctr;          // kCtr*
  uint32_t* cb;           // [T - 1][6] centroid bounds (encoded) of the block task at each node slot
  float4* nodes;
  uint32_t* child;
  uint32_t* parent;
  float* nbox;
  uint32_t* misc;
  uint32_t n;
};

__device__ __forceinline__ float box_area_rn(float3 lo, float3 hi) {
  const float dx = __fsub_rn(hi.x, lo.x), dy = __fsub_rn(hi.y, lo.y), dz = __fsub_rn(hi.z, lo.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dy), __fmul_rn(dy, dz)), __fmul_rn(dz, dx));
}
__device__ __forceinline__ float3 cl_centroid(float4 lo, float4 hi) {
  return make_float3(__fmul_rn(0.5f, __fadd_rn(lo.x, hi.x)), __fmul_rn(0.5f, __fadd_rn(lo.y, hi.y)),
                     __fmul_rn(0.5f, __fadd_rn(lo.z, hi.z)));
}
__device__ __forceinline__ int top_bin(float c, float cmin, float scale) {
  return min(__float2int_rz(__fmul_rn(__fsub_rn(c, cmin), scale)), kTopBins - 1);
}
__device__ __forceinline__ float comp(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

constexpr uint32_t kEncPosInf = 0xFF800000u, kEncNegInf = 0x007FFFFFu;   // enc_f(+inf), enc_f(-inf)
constexpr int kBinWords = 8;   // per bin: clusters, weight, lo xyz, hi xyz (encoded)
constexpr int kTopItems = 2;   // records per thread per round of a block pass
constexpr int kBinCopy = 3 * kTopBins * kBinWords + 1;   // words per copy of a block task's bins (+1: copies in different banks)

__device__ __forceinline__ void bins_clear(uint32_t* bins, int i0, int stride) {
  for (int i = i0; i < 3 * kTopBins; i += stride) {
    uint32_t* q = bins + kBinWords * i;
    q[0] = 0u;
    q[1] = 0u;
    q[2] = q[3] = q[4] = kEncPosInf;
    q[5] = q[6] = q[7] = kEncNegInf;
  }
}
struct Split {
  bool valid;
  float cost;
  int q;
  uint32_t nl;   // clusters left of the split
};

// Best split after one of the bins of one axis (bins: [kTopBins][kBinWords]),
// evaluated by a full warp, lane q = bin q, with prefix (left) and suffix
// (right) sweeps; the result is the same in every lane.  Lowest cost, ties
// to the lower bin.
__device__ Split warp_best_split(const uint32_t* bins, int lane) {
  const uint32_t* b = bins + kBinWords * lane;
  uint32_t pn = b[0], pw = b[1];
  float3 plo = make_float3(dec_f(b[2]), dec_f(b[3]), dec_f(b[4]));
  float3 phi = make_float3(dec_f(b[5]), dec_f(b[6]), dec_f(b[7]));
  uint32_t sn = pn, sw = pw;
  float3 slo = plo, shi = phi;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t yn = __shfl_up_sync(0xFFFFFFFFu, pn, off), yw = __shfl_up_sync(0xFFFFFFFFu, pw, off);
    const float ylx = __shfl_up_sync(0xFFFFFFFFu, plo.x, off), yly = __shfl_up_sync(0xFFFFFFFFu, plo.y, off),
                ylz = __shfl_up_sync(0xFFFFFFFFu, plo.z, off);
    const float yhx = __shfl_up_sync(0xFFFFFFFFu, phi.x, off), yhy = __shfl_up_sync(0xFFFFFFFFu, phi.y, off),
                yhz = __shfl_up_sync(0xFFFFFFFFu, phi.z, off);
    const uint32_t zn = __shfl_down_sync(0xFFFFFFFFu, sn, off), zw = __shfl_down_sync(0xFFFFFFFFu, sw, off);
    const float zlx = __shfl_down_sync(0xFFFFFFFFu, slo.x, off), zly = __shfl_down_sync(0xFFFFFFFFu, slo.y, off),
                zlz = __shfl_down_sync(0xFFFFFFFFu, slo.z, off);
    const float zhx = __shfl_down_sync(0xFFFFFFFFu, shi.x, off), zhy = __shfl_down_sync(0xFFFFFFFFu, shi.y, off),
                zhz = __shfl_down_sync(0xFFFFFFFFu, shi.z, off);
    if (lane >= off) {
      pn += yn;
      pw += yw;
      plo = make_float3(fminf(plo.x, ylx), fminf(plo.y, yly), fminf(plo.z, ylz));
      phi = make_float3(fmaxf(phi.x, yhx), fmaxf(phi.y, yhy), fmaxf(phi.z, yhz));
    }
    if (lane + off < 32) {
      sn += zn;
      sw += zw;
      slo = make_float3(fminf(slo.x, zlx), fminf(slo.y, zly), fminf(slo.z, zlz));
      shi = make_float3(fmaxf(shi.x, zhx), fmaxf(shi.y, zhy), fmaxf(shi.z, zhz));
    }
  }
  // split after bin lane - 1: left = prefix of lane - 1, right = suffix of lane
  const uint32_t ln = __shfl_up_sync(0xFFFFFFFFu, pn, 1), lw = __shfl_up_sync(0xFFFFFFFFu, pw, 1);
  const float llx = __shfl_up_sync(0xFFFFFFFFu, plo.x, 1), lly = __shfl_up_sync(0xFFFFFFFFu, plo.y, 1),
              llz = __shfl_up_sync(0xFFFFFFFFu, plo.z, 1);
  const float lhx = __shfl_up_sync(0xFFFFFFFFu, phi.x, 1), lhy = __shfl_up_sync(0xFFFFFFFFu, phi.y, 1),
              lhz = __shfl_up_sync(0xFFFFFFFFu, phi.z, 1);
  Split r;
  r.valid = lane >= 1 && ln > 0u && sn > 0u;
  r.cost = 0.0f;
  r.q = lane;
  r.nl = ln;
  if (r.valid) {
    const float al = box_area_rn(make_float3(llx, lly, llz), make_float3(lhx, lhy, lhz));
    const float ar = box_area_rn(slo, shi);
    r.cost = __fadd_rn(__fmul_rn(al, __uint2float_rn(lw)), __fmul_rn(ar, __uint2float_rn(sw)));
  }
  for (int off = 16; off > 0; off >>= 1) {
    const bool ov = __shfl_xor_sync(0xFFFFFFFFu, r.valid, off);
    const float oc = __shfl_xor_sync(0xFFFFFFFFu, r.cost, off);
    const int oq = __shfl_xor_sync(0xFFFFFFFFu, r.q, off);
    const uint32_t onl = __shfl_xor_sync(0xFFFFFFFFu, r.nl, off);
    if (ov && (!r.valid || oc < r.cost || (oc == r.cost && oq < r.q))) {
      r.valid = true;
      r.cost = oc;
      r.q = oq;
      r.nl = onl;
    }
  }
  return r;
}

// the node of a task: child boxes (lo xyz, hi xyz) and references
__device__ __forceinline__ void write_top_node(const TopArgs& a, uint32_t slot, const float (&bx)[2][6],
                                               const uint32_t (&ref)[2]) {
  float4* nd = a.nodes + 4 * (size_t)slot;
  nd[0] = make_float4(bx[0][0], bx[0][3], bx[0][1], bx[0][4]);
  nd[1] = make_float4(bx[1][0], bx[1][3], bx[1][1], bx[1][4]);
  nd[2] = make_float4(bx[0][2], bx[0][5], bx[1][2], bx[1][5]);
  nd[3] = make_float4(__uint_as_float(ref[0]), __uint_as_float(ref[1]), 0.f, 0.f);
  a.child[2 * slot] = ref[0];
  a.child[2 * slot + 1] = ref[1];
  for (int side = 0; side < 2; ++side) a.parent[node_slot(ref[side], a.n)] = slot;
  float* nb = a.nbox + 6 * (size_t)slot;
  for (int q = 0; q < 3; ++q) {
    nb[q] = fminf(bx[0][q], bx[1][q]);
    nb[3 + q] = fmaxf(bx[0][3 + q], bx[1][3 + q]);
  }
}

// Block tasks (more than kTopSmall clusters), persistent: each block takes
// the next task number and waits (bounded) until that task is published.
// Tasks are numbered in the order they are created, a task by the block
// working on its parent, which took a smaller number earlier and is running;
// so the smallest number any block waits for belongs to a parent in
// progress, and every wait ends -- with the task, or with the count of
// pending tasks at zero when no task of that number will come.  A block
// goes on with one large child itself (no number, no wait; it stays counted
// as pending), publishes the other; children of at most kTopSmall clusters
// go to the warp-task list.  The cluster records move with the partition, so
// every pass reads its task's records contiguously, kTopItems per thread.
__global__ void __launch_bounds__(kTopBlock) k_top_sah(TopArgs a) {
  __shared__ uint32_t s_bins[8][kBinCopy];   // one copy per lane mod 8, summed into [0]
  __shared__ uint32_t s_cb[6], s_side[2][6], s_cside[2][6];
  __shared__ uint32_t s_task[4], s_stop, s_cont;
  __shared__ Split s_split[3];
  __shared__ uint32_t s_wl[2][kTopBlock / 32], s_wr[2][kTopBlock / 32];   // by round parity
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t C = a.ctr[kCtrClusters];
  if (C <= kTopSmall) return;   // no block task: the warp tasks do it all
  const uint32_t n_nodes = C - 1;
  if (a.ctr[kCtrMarked] + 1u != n_nodes) {   // the marked top part and the clusters disagree: leave the LBVH as it is
    if (blockIdx.x == 0 && tid == 0) atomicOr(&a.misc[6], kErrTopBuild);
    return;
  }
  if (tid == 0) s_cont = 0u;
  __syncthreads();
  while (true) {
    if (tid == 0 && !s_cont) {
      s_stop = 0u;
      const uint32_t ti = atomicAdd(&a.ctr[kCtrHead], 1u);
      if (ti >= n_nodes) {
        s_stop = 1u;
      } else {
        // poll the own flag; the shared counters only now and then, so that
        // waiting blocks do not crowd the lines the working blocks update
        uint32_t spins = 0, nap = 32;
        while (ld_acquire_u32(&a.ready[ti]) == 0u) {
          if ((spins & 15u) == 15u) {
            if (ld_acquire_u32(&a.ctr[kCtrPending]) == 0u) {   // all tasks done: none numbered ti will come
              s_stop = 1u;
              break;
            }
            if (ld_acquire_u32(&a.misc[6]) & kErrTopBuild) {
              s_stop = 1u;
              break;
            }
          }
          if (++spins > kTopSpinLimit) {
            atomicOr(&a.misc[6], kErrTopBuild);
            s_stop = 1u;
            break;
          }
          __nanosleep(nap);
          if (nap < 256) nap <<= 1;
        }
        if (!s_stop) {
          const uint4 t = __ldcg(&a.task[ti]);
          s_task[0] = t.x;
          s_task[1] = t.y;
          s_task[2] = t.z;
          s_task[3] = t.w;
        }
      }
    }
    if (tid == 0 && (s_cont || !s_stop))
      for (int q = 0; q < 6; ++q) s_cb[q] = __ldcg(&a.cb[6 * (size_t)s_task[2] + q]);
    __syncthreads();
    if (!s_cont && s_stop) return;
    const uint32_t b = s_task[0], n = s_task[1] - s_task[0], slot = s_task[2];
    const uint32_t depth = s_task[3] & 0x7FFFFFFFu, src = s_task[3] >> 31;
    const float4* in = a.rec[src] + 2 * (size_t)b;
    float4* out = a.rec[src ^ 1u] + 2 * (size_t)b;
    for (int w = 0; w < 8; ++w) bins_clear(s_bins[w], tid, kTopBlock);
    if (tid < 6) {
      s_side[0][tid] = s_cside[0][tid] = tid < 3 ? kEncPosInf : kEncNegInf;
      s_side[1][tid] = s_cside[1][tid] = tid < 3 ? kEncPosInf : kEncNegInf;
    }
    __syncthreads();
    float cmin[3], scale[3];
    bool axis_ok[3];
    for (int k = 0; k < 3; ++k) {
      cmin[k] = dec_f(s_cb[k]);
      const float ext = __fsub_rn(dec_f(s_cb[3 + k]), cmin[k]);
      axis_ok[k] = ext > 0.0f && depth < kTopMedianDepth;
      scale[k] = axis_ok[k] ? __fdiv_rn((float)kTopBins, ext) : 0.0f;
    }
    // bins: each thread takes a contiguous chunk of the task (Morton order,
    // so neighbours mostly share bins) and adds runs of one bin at a time to
    // the copy of its lane mod 8: the lanes of a warp hold neighbouring chunks,
    // mostly in the same bins, and same-address shared atomics of one warp
    // serialise, so at most 4 lanes share an address
    if (axis_ok[0] || axis_ok[1] || axis_ok[2]) {
      int run_q[3] = {-1, -1, -1};
      uint32_t run_n[3] = {0u, 0u, 0u}, run_w[3] = {0u, 0u, 0u};
      float run_b[3][6];
      const uint32_t chunk = (n + kTopBlock - 1) / kTopBlock;
      const uint32_t i0 = min(n, chunk * tid), i1 = min(n, i0 + chunk);
      for (uint32_t ib = i0; ib < i1; ib += kTopItems) {
        float4 blo[kTopItems], bhi[kTopItems];
#pragma unroll
        for (int k = 0; k < kTopItems; ++k)
          if (ib + k < i1) {
            blo[k] = __ldcg(in + 2 * (ib + k));
            bhi[k] = __ldcg(in + 2 * (ib + k) + 1);
          }
#pragma unroll
        for (int k = 0; k < kTopItems; ++k) {
          if (ib + k >= i1) break;
          const float4 lo = blo[k], hi = bhi[k];
          const float3 cc = cl_centroid(lo, hi);
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) {
            if (!axis_ok[ax]) continue;
            const int q = top_bin(comp(cc, ax), cmin[ax], scale[ax]);
            if (q != run_q[ax]) {
              if (run_q[ax] >= 0) {
                uint32_t* bb = s_bins[lane & 7] + kBinWords * (ax * kTopBins + run_q[ax]);
                atomicAdd(&bb[0], run_n[ax]);
                atomicAdd(&bb[1], run_w[ax]);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  atomicMin(&bb[2 + c], enc_f(run_b[ax][c]));
                  atomicMax(&bb[5 + c], enc_f(run_b[ax][3 + c]));
                }
              }
              run_q[ax] = q;
              run_n[ax] = 0u;
              run_w[ax] = 0u;
              run_b[ax][0] = run_b[ax][1] = run_b[ax][2] = INFINITY;
              run_b[ax][3] = run_b[ax][4] = run_b[ax][5] = -INFINITY;
            }
            ++run_n[ax];
            run_w[ax] += __float_as_uint(lo.w);
            run_b[ax][0] = fminf(run_b[ax][0], lo.x);
            run_b[ax][1] = fminf(run_b[ax][1], lo.y);
            run_b[ax][2] = fminf(run_b[ax][2], lo.z);
            run_b[ax][3] = fmaxf(run_b[ax][3], hi.x);
            run_b[ax][4] = fmaxf(run_b[ax][4], hi.y);
            run_b[ax][5] = fmaxf(run_b[ax][5], hi.z);
          }
        }
      }
#pragma unroll
      for (int ax = 0; ax < 3; ++ax)
        if (run_q[ax] >= 0) {
          uint32_t* bb = s_bins[lane & 7] + kBinWords * (ax * kTopBins + run_q[ax]);
          atomicAdd(&bb[0], run_n[ax]);
          atomicAdd(&bb[1], run_w[ax]);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            atomicMin(&bb[2 + c], enc_f(run_b[ax][c]));
            atomicMax(&bb[5 + c], enc_f(run_b[ax][3 + c]));
          }
        }
    }
    __syncthreads();
    // the lanes' copies into copy 0: sums of counts and weights, min / max of
    // the (order-preserving) encoded bounds
    for (int i = tid; i < 3 * kTopBins * kBinWords; i += kTopBlock) {
      const int word = i % kBinWords;
      uint32_t v = s_bins[0][i];
      for (int w = 1; w < 8; ++w) {
        const uint32_t u = s_bins[w][i];
        v = word < 2 ? v + u : (word < 5 ? min(v, u) : max(v, u));
      }
      s_bins[0][i] = v;
    }
    __syncthreads();
    if (warp < 3) {
      Split r;
      r.valid = false;
      if (axis_ok[warp]) r = warp_best_split(s_bins[0] + kBinWords * kTopBins * warp, lane);
      if (lane == 0) s_split[warp] = r;
    }
    __syncthreads();
    int axis = -1, split = 0;
    uint32_t nl = n / 2u;
    for (int k = 0; k < 3; ++k)
      if (s_split[k].valid && (axis < 0 || s_split[k].cost < s_split[axis].cost)) axis = k;
    if (axis >= 0) {
      split = s_split[axis].q;
      nl = s_split[axis].nl;
    }
    const float a_min = axis == 0 ? cmin[0] : (axis == 1 ? cmin[1] : cmin[2]);
    const float a_scale = axis == 0 ? scale[0] : (axis == 1 ? scale[1] : scale[2]);
    // stable partition of the records into the other buffer; each thread
    // keeps its sides' boxes and centroid bounds over all rounds, reduced once
    float v[2][6] = {{INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY},
                     {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY}};
    float cv[2][6] = {{INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY},
                      {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY}};
    // one barrier a round: the warps' counts are kept by round parity, and
    // every thread keeps the running offsets of both sides itself
    uint32_t base_l = 0u, base_r = 0u, rnd = 0u;
    for (uint32_t t0 = 0; t0 < n; t0 += kTopItems * kTopBlock, ++rnd) {
      const uint32_t i0 = t0 + kTopItems * tid;
      float4 lo[kTopItems], hi[kTopItems];
      uint32_t lmask = 0u, hmask = 0u;
#pragma unroll
      for (int k = 0; k < kTopItems; ++k)
        if (i0 + k < n) {
          lo[k] = __ldcg(in + 2 * (i0 + k));
          hi[k] = __ldcg(in + 2 * (i0 + k) + 1);
        }
#pragma unroll
      for (int k = 0; k < kTopItems; ++k) {
        const uint32_t i = i0 + k;
        if (i < n) {
          const float3 cc = cl_centroid(lo[k], hi[k]);
          const bool left = axis >= 0 ? top_bin(comp(cc, axis), a_min, a_scale) < split : i < nl;
          hmask |= 1u << k;
          if (left) lmask |= 1u << k;
          // both sides' accumulators by select: static indices keep them in registers
#pragma unroll
          for (int sd = 0; sd < 2; ++sd) {
            const bool on = left == (sd == 0);
            const float inf = INFINITY;
            v[sd][0] = fminf(v[sd][0], on ? lo[k].x : inf);
            v[sd][1] = fminf(v[sd][1], on ? lo[k].y : inf);
            v[sd][2] = fminf(v[sd][2], on ? lo[k].z : inf);
            v[sd][3] = fmaxf(v[sd][3], on ? hi[k].x : -inf);
            v[sd][4] = fmaxf(v[sd][4], on ? hi[k].y : -inf);
            v[sd][5] = fmaxf(v[sd][5], on ? hi[k].z : -inf);
            cv[sd][0] = fminf(cv[sd][0], on ? cc.x : inf);
            cv[sd][1] = fminf(cv[sd][1], on ? cc.y : inf);
            cv[sd][2] = fminf(cv[sd][2], on ? cc.z : inf);
            cv[sd][3] = fmaxf(cv[sd][3], on ? cc.x : -inf);
            cv[sd][4] = fmaxf(cv[sd][4], on ? cc.y : -inf);
            cv[sd][5] = fmaxf(cv[sd][5], on ? cc.z : -inf);
          }
        }
      }
      const uint32_t cl = __popc(lmask), cr = __popc(hmask & ~lmask);
      // exclusive offsets of the threads' left and right counts
      uint32_t xl = cl, xr = cr;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t yl = __shfl_up_sync(0xFFFFFFFFu, xl, off), yr = __shfl_up_sync(0xFFFFFFFFu, xr, off);
        if (lane >= off) {
          xl += yl;
          xr += yr;
        }
      }
      const uint32_t par = rnd & 1u;
      if (lane == 31) {
        s_wl[par][warp] = xl;
        s_wr[par][warp] = xr;
      }
      __syncthreads();
      uint32_t offl = base_l + xl - cl, offr = base_r + xr - cr, totl = 0, totr = 0;
      for (int w = 0; w < kTopBlock / 32; ++w) {
        const uint32_t wl = s_wl[par][w], wr = s_wr[par][w];
        if (w < warp) {
          offl += wl;
          offr += wr;
        }
        totl += wl;
        totr += wr;
      }
#pragma unroll
      for (int k = 0; k < kTopItems; ++k) {
        if (!(hmask >> k & 1u)) continue;
        const bool left = lmask >> k & 1u;   // (k is static here: the records stay in registers)
        // the bins and this pass classify with the same arithmetic, so the
        // left side holds exactly nl clusters; refuse anything else
        const uint32_t pos = left ? offl++ : nl + offr++;
        if (left ? pos < nl : pos < n) {
          out[2 * pos] = lo[k];
          out[2 * pos + 1] = hi[k];
        } else {
          atomicOr(&a.misc[6], kErrTopBuild);
        }
      }
      base_l += totl;
      base_r += totr;
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const float o = __shfl_xor_sync(0xFFFFFFFFu, v[side][q], off);
          const float oc = __shfl_xor_sync(0xFFFFFFFFu, cv[side][q], off);
          v[side][q] = q < 3 ? fminf(v[side][q], o) : fmaxf(v[side][q], o);
          cv[side][q] = q < 3 ? fminf(cv[side][q], oc) : fmaxf(cv[side][q], oc);
        }
      if (lane == 0 && v[side][0] <= v[side][3])
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          if (q < 3) {
            atomicMin(&s_side[side][q], enc_f(v[side][q]));
            atomicMin(&s_cside[side][q], enc_f(cv[side][q]));
          } else {
            atomicMax(&s_side[side][q], enc_f(v[side][q]));
            atomicMax(&s_cside[side][q], enc_f(cv[side][q]));
          }
        }
    }
    __threadfence();   // the new order is visible before the children are published
    __syncthreads();
    if (tid == 0) {
      uint32_t ref[2] = {kNone, kNone}, pend[2] = {kNone, kNone}, n_pend = 0;
      bool ok = true, cont = false;
      uint4 next = make_uint4(0u, 0u, 0u, 0u);
      // what each side needs: a leaf reference, a node and a warp task, or a
      // node and a block task (the first large side continues in this block)
      const uint32_t cnt[2] = {nl, n - nl}, first[2] = {0u, nl};
      uint32_t n_int = 0, n_sm = 0, n_big = 0;
      int keep = -1;
      for (int side = 0; side < 2; ++side) {
        if (cnt[side] < 2u) continue;
        ++n_int;
        if (cnt[side] <= kTopSmall) ++n_sm;
        else if (keep < 0) keep = side;
        else ++n_big;
      }
      // independent counter updates, in flight together
      const uint32_t sbase = n_int ? 1u + atomicAdd(&a.ctr[kCtrSlots], n_int) : 0u;
      const uint32_t mbase = n_sm ? atomicAdd(&a.ctr[kCtrSmall], n_sm) : 0u;
      const uint32_t tbase = n_big ? atomicAdd(&a.ctr[kCtrTasks], n_big) : 0u;
      // cannot fail for a consistent marking; refuse rather than write past the arrays
      ok = sbase + n_int <= n_nodes && mbase + n_sm <= n_nodes && tbase + n_big <= n_nodes;
      uint32_t k_int = 0, k_sm = 0, k_big = 0;
      for (int side = 0; side < 2 && ok; ++side) {
        if (cnt[side] == 1u) {
          ref[side] = __float_as_uint(__ldcg(out + 2 * first[side] + 1).w);
          continue;
        }
        ref[side] = a.slot[sbase + k_int++];
        const uint4 t = make_uint4(b + first[side], b + first[side] + cnt[side], ref[side],
                                   (depth + 1u) | ((src ^ 1u) << 31));
        if (cnt[side] > kTopSmall)
          for (int q = 0; q < 6; ++q) a.cb[6 * (size_t)ref[side] + q] = s_cside[side][q];
        if (side == keep) {   // this block goes on with it
          cont = true;
          next = t;
        } else if (cnt[side] <= kTopSmall) {
          a.small[mbase + k_sm++] = t;
        } else {
          pend[side] = tbase + k_big++;
          a.task[pend[side]] = t;
          ++n_pend;
        }
      }
      if (!ok) {
        atomicOr(&a.misc[6], kErrTopBuild);
        cont = false;
      } else {
        float bx[2][6];
        for (int side = 0; side < 2; ++side)
          for (int q = 0; q < 6; ++q) bx[side][q] = dec_f(s_side[side][q]);
        write_top_node(a, slot, bx, ref);
        if (n_pend) atomicAdd(&a.ctr[kCtrPending], n_pend);   // counted before they can finish
        __threadfence();
        for (int side = 0; side < 2; ++side)
          if (pend[side] != kNone) st_release_u32(&a.ready[pend[side]], 1u);
      }
      if (cont) {   // still pending: the task continues as its child
        s_task[0] = next.x;
        s_task[1] = next.y;
        s_task[2] = next.z;
        s_task[3] = next.w;
        s_cont = 1u;
      } else {
        s_cont = 0u;
        atomicSub(&a.ctr[kCtrPending], 1u);   // this task is done
      }
    }
    __syncthreads();
  }
}

// Warp tasks (2 to kTopSmall clusters), after the block tasks: a warp builds
// the whole subtree of a task, a cluster per lane, one tree level at a time.
// The sub-tasks of a level are disjoint sets of lanes (segments, kept as lane
// masks; the lane order is the cluster order, so splitting a mask keeps the
// order on both sides), and all of them are worked at once: each lane
// evaluates, for its own segment, the split after its own bin on every axis
// -- a partition {bin < q} is reached first (lowest q) at q = 1 + the largest
// bin on its left, so these are exactly the splits the bin sweep of a block
// task can choose, each with its lowest q -- and the segment takes the lowest
// (cost, axis, q).  The same rules and arithmetic as the block tasks.
constexpr int kSmallWarps = 8;
__global__ void __launch_bounds__(32 * kSmallWarps) k_top_small(TopArgs a) {
  __shared__ float4 s_rec[kSmallWarps][kTopSmall][2];     // (lo xyz, weight) (hi xyz, reference)
  __shared__ uint32_t s_bin[kSmallWarps][kTopSmall];     // the three bins, 8 bits each
  __shared__ float s_cost[kSmallWarps][kTopSmall];
  __shared__ uint32_t s_key[kSmallWarps][kTopSmall];   // valid << 31 | nl << 10 | axis << 8 | q
  __shared__ uint32_t s_slot[kSmallWarps][kTopSmall], s_child[kSmallWarps][kTopSmall][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t C = a.ctr[kCtrClusters];
  if (C < 2 || (a.misc[6] & kErrTopBuild)) return;
  if (a.ctr[kCtrMarked] + 2u != C) {   // the marked top part and the clusters disagree: leave the LBVH as it is
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.misc[6], kErrTopBuild);
    return;
  }
  const uint32_t n_nodes = C - 1, n_small = min(a.ctr[kCtrSmall], n_nodes);
  while (true) {
    uint32_t si = 0;
    if (lane == 0) si = atomicAdd(&a.ctr[kCtrSmallHead], 1u);
    si = __shfl_sync(0xFFFFFFFFu, si, 0);
    if (si >= n_small) return;
    const uint4 t = a.small[si];
    const uint32_t n = t.y - t.x;
    if (n < 2u || n > kTopSmall) {   // cannot happen: only such tasks are listed
      if (lane == 0) atomicOr(&a.misc[6], kErrTopBuild);
      return;
    }
    const bool mine = (uint32_t)lane < n;
    const float4* in = a.rec[t.w >> 31] + 2 * (size_t)t.x;
    const float4 lo = mine ? __ldcg(in + 2 * lane) : make_float4(INFINITY, INFINITY, INFINITY, 0.f);
    const float4 hi = mine ? __ldcg(in + 2 * lane + 1) : make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
    const float3 cc = cl_centroid(lo, hi);
    s_rec[warp][lane][0] = lo;
    s_rec[warp][lane][1] = hi;
    // the subtree of n clusters has n - 1 internal nodes; its root has its slot
    uint32_t sbase = 0;
    if (lane == 0 && n > 2u) sbase = 1u + atomicAdd(&a.ctr[kCtrSlots], n - 2u);
    sbase = __shfl_sync(0xFFFFFFFFu, sbase, 0);
    if (n > 2u && sbase + (n - 2u) > n_nodes) {   // cannot happen for a consistent marking
      if (lane == 0) atomicOr(&a.misc[6], kErrTopBuild);
      return;
    }
    if ((uint32_t)lane + 2u < n) s_slot[warp][lane] = a.slot[sbase + lane];
    uint32_t next_slot = 0;   // new nodes taken so far (warp-uniform)
    // the lane's segment (0: none, or a single cluster), its node slot and depth
    uint32_t seg = mine ? (n == 32u ? 0xFFFFFFFFu : (1u << n) - 1u) : 0u;
    uint32_t seg_slot = t.z, depth = t.w & 0x7FFFFFFFu;
    __syncwarp();
    bool fail = false;
    while (true) {
      const bool act = __popc(seg) >= 2;
      if (!__any_sync(0xFFFFFFFFu, act)) break;
      // segment centroid bounds, bins
      float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (uint32_t m = act ? seg : 0u; m; m &= m - 1u) {
        const int j = __ffs(m) - 1;
        const float3 cj = cl_centroid(s_rec[warp][j][0], s_rec[warp][j][1]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          mn[k] = fminf(mn[k], comp(cj, k));
          mx[k] = fmaxf(mx[k], comp(cj, k));
        }
      }
      bool axis_ok[3];
      int my_bin[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float ext = __fsub_rn(mx[k], mn[k]);
        axis_ok[k] = act && ext > 0.0f && depth < kTopMedianDepth;
        my_bin[k] = axis_ok[k] ? top_bin(comp(cc, k), mn[k], __fdiv_rn((float)kTopBins, ext)) : kTopBins;
      }
      s_bin[warp][lane] = (uint32_t)my_bin[0] | ((uint32_t)my_bin[1] << 8) | ((uint32_t)my_bin[2] << 16);
      __syncwarp();
      // this lane's best split over the axes: lowest cost, ties to the lower axis;
      // the split after the lane's own bin on each axis, all three in one pass
      // over the segment's members
      bool valid = false;
      float cost = 0.0f;
      int b_axis = 0, b_q = 0;
      uint32_t b_nl = 0;
      if (act && (axis_ok[0] || axis_ok[1] || axis_ok[2])) {
        float3 llo[3], lhi[3], rlo[3], rhi[3];
        uint32_t lw[3], rw[3], lc[3], rc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          llo[k] = rlo[k] = make_float3(INFINITY, INFINITY, INFINITY);
          lhi[k] = rhi[k] = make_float3(-INFINITY, -INFINITY, -INFINITY);
          lw[k] = rw[k] = lc[k] = rc[k] = 0u;
        }
        for (uint32_t m = seg; m; m &= m - 1u) {
          const int j = __ffs(m) - 1;
          const float4 jlo = s_rec[warp][j][0], jhi = s_rec[warp][j][1];
          const uint32_t jb = s_bin[warp][j], wj = __float_as_uint(jlo.w);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const bool lft = (int)((jb >> (8 * k)) & 0xFFu) <= my_bin[k];   // bin < my_bin + 1
            if (lft) {
              llo[k] = make_float3(fminf(llo[k].x, jlo.x), fminf(llo[k].y, jlo.y), fminf(llo[k].z, jlo.z));
              lhi[k] = make_float3(fmaxf(lhi[k].x, jhi.x), fmaxf(lhi[k].y, jhi.y), fmaxf(lhi[k].z, jhi.z));
              lw[k] += wj;
              ++lc[k];
            } else {
              rlo[k] = make_float3(fminf(rlo[k].x, jlo.x), fminf(rlo[k].y, jlo.y), fminf(rlo[k].z, jlo.z));
              rhi[k] = make_float3(fmaxf(rhi[k].x, jhi.x), fmaxf(rhi[k].y, jhi.y), fmaxf(rhi[k].z, jhi.z));
              rw[k] += wj;
              ++rc[k];
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if (!axis_ok[k] || lc[k] == 0u || rc[k] == 0u) continue;
          const float c = __fadd_rn(__fmul_rn(box_area_rn(llo[k], lhi[k]), __uint2float_rn(lw[k])),
                                    __fmul_rn(box_area_rn(rlo[k], rhi[k]), __uint2float_rn(rw[k])));
          if (!valid || c < cost) {
            valid = true;
            cost = c;
            b_axis = k;
            b_q = my_bin[k] + 1;
            b_nl = lc[k];
          }
        }
      }
      s_cost[warp][lane] = cost;
      s_key[warp][lane] = (valid ? 0x80000000u : 0u) | (b_nl << 10) | ((uint32_t)b_axis << 8) | (uint32_t)b_q;
      __syncwarp();
      // the segment's split: lowest (cost, axis, q) over its lanes
      bool s_valid = false;
      float s_c = 0.0f;
      uint32_t s_k = 0;
      for (uint32_t m = act ? seg : 0u; m; m &= m - 1u) {
        const int j = __ffs(m) - 1;
        const uint32_t key = s_key[warp][j];
        if (!(key & 0x80000000u)) continue;
        const float c = s_cost[warp][j];
        if (!s_valid || c < s_c || (c == s_c && (key & 0x3FFu) < (s_k & 0x3FFu))) {
          s_valid = true;
          s_c = c;
          s_k = key;
        }
      }
      const uint32_t n_seg = __popc(seg);
      const int axis = s_valid ? (int)((s_k >> 8) & 3u) : -1;
      const int split = (int)(s_k & 0xFFu);
      const uint32_t nl = s_valid ? (s_k >> 10) & 0x3Fu : n_seg / 2u;
      const int a_bin = axis == 0 ? my_bin[0] : (axis == 1 ? my_bin[1] : my_bin[2]);
      const bool left = act && (axis >= 0 ? a_bin < split : (uint32_t)__popc(seg & lt) < nl);
      const uint32_t lmask = __ballot_sync(0xFFFFFFFFu, left);
      const uint32_t lseg = seg & lmask, rseg = seg & ~lmask;
      if (act && ((uint32_t)__popc(lseg) != nl || lseg == 0u || rseg == 0u)) fail = true;   // cannot happen
      if (__any_sync(0xFFFFFFFFu, fail)) {
        fail = true;
        break;
      }
      // the segment's leader (its lowest lane) writes the node; new nodes take
      // slots in lane order of their leaders
      const bool leader = act && (seg & lt) == 0u;
      const uint32_t need = leader ? (uint32_t)(__popc(lseg) >= 2) + (uint32_t)(__popc(rseg) >= 2) : 0u;
      uint32_t x = need;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if (lane >= off) x += y;
      }
      const uint32_t total = __shfl_sync(0xFFFFFFFFu, x, 31);
      if (next_slot + total + 2u > n) fail = true;   // cannot happen: n - 2 new nodes at most
      if (__any_sync(0xFFFFFFFFu, fail)) {
        fail = true;
        break;
      }
      if (leader) {
        uint32_t k_new = next_slot + x - need;
        float bx[2][6];
        uint32_t ref[2];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const uint32_t sm = side ? rseg : lseg;
          float v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
          for (uint32_t m = sm; m; m &= m - 1u) {
            const float4 jlo = s_rec[warp][__ffs(m) - 1][0], jhi = s_rec[warp][__ffs(m) - 1][1];
            v[0] = fminf(v[0], jlo.x);
            v[1] = fminf(v[1], jlo.y);
            v[2] = fminf(v[2], jlo.z);
            v[3] = fmaxf(v[3], jhi.x);
            v[4] = fmaxf(v[4], jhi.y);
            v[5] = fmaxf(v[5], jhi.z);
          }
          for (int q = 0; q < 6; ++q) bx[side][q] = v[q];
          ref[side] = __popc(sm) == 1 ? __float_as_uint(s_rec[warp][__ffs(sm) - 1][1].w) : s_slot[warp][k_new++];
          s_child[warp][lane][side] = ref[side];
        }
        write_top_node(a, seg_slot, bx, ref);
      }
      next_slot += total;
      __syncwarp();
      if (act) {   // into the own half: its node (from the leader), one level deeper
        const uint32_t half = left ? lseg : rseg;
        seg_slot = s_child[warp][__ffs(seg) - 1][left ? 0 : 1];
        seg = __popc(half) >= 2 ? half : 0u;
        ++depth;
      }
      __syncwarp();
    }
    if (fail) {
      if (lane == 0) atomicOr(&a.misc[6], kErrTopBuild);
      return;
    }
  }
}

// ---------------------------------------------------------------------------
// lobe tables: cell integrals of cos^C by 8-point Gauss-Legendre, then a
// compensated prefix per material
// ---------------------------------------------------------------------------
// a6: 8-wide BVH with 8-bit quantised child boxes, collapsed from the binary
// LBVH (wide node layout in rr_internal.cuh).
//
// A: every binary internal node b computes the cut it would have as the root
//    of a wide node: starting from its two children, the internal member of
//    largest surface area is replaced by its two children until there are 8
//    members or only leaves.  Members get slots by octant: slot bit k is set
//    when the member lies on the high side of axis k (greedy assignment by
//    the centroid offset from the node centre), so that a ray visiting slots
//    in the order k ^ octant(direction) meets near members first.
__device__ __forceinline__ float box_area(const float* b) {
  const float dx = b[3] - b[0], dy = b[4] - b[1], dz = b[5] - b[2];
  return dx * dy + dy * dz + dz * dx;
}

__global__ void k_wide_cut(uint32_t n, const uint32_t* __restrict__ child, const float* __restrict__ nbox,
                           uint32_t* __restrict__ cut, uint32_t* __restrict__ wctr) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) {   // counters of pass B: ticket, allocated (the root), done, triangles, error
    wctr[0] = 0u;
    wctr[1] = 1u;
    wctr[2] = 0u;
    wctr[3] = 0u;
    wctr[4] = 0u;
  }
  if (b + 1 >= n) return;
  uint32_t c[8];
  float bx[8][6];
  c[0] = classify_member(__ldg(&child[2 * b]), child);
  c[1] = classify_member(__ldg(&child[2 * b + 1]), child);
  int m = 2;
  for (int k = 0; k < 2; ++k)
    for (int q = 0; q < 6; ++q) bx[k][q] = __ldg(&nbox[6 * (size_t)member_box(c[k], n) + q]);
  // open the largest inner member while a slot is free; once only leaves and
  // groups are left, open the largest group (tighter boxes in the free slots)
  while (m < 8) {
    int best = -1;
    float best_a = -1.0f;
    for (int pass = 0; pass < 2 && best < 0; ++pass)
      for (int k = 0; k < m; ++k) {
        if (pass == 0 ? !member_is_inner(c[k]) : !member_is_group(c[k])) continue;
        const float a = box_area(bx[k]);
        if (a > best_a) {
          best_a = a;
          best = k;
        }
      }
    if (best < 0) break;
    const uint32_t p = c[best] & kGroupNodeMask;
    const uint32_t c0 = classify_member(__ldg(&child[2 * p]), child);
    const uint32_t c1 = classify_member(__ldg(&child[2 * p + 1]), child);
    c[best] = c0;
    c[m] = c1;
    for (int q = 0; q < 6; ++q) {
      bx[best][q] = __ldg(&nbox[6 * (size_t)member_box(c0, n) + q]);
      bx[m][q] = __ldg(&nbox[6 * (size_t)member_box(c1, n) + q]);
    }
    ++m;
  }
  // octant slots
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int k = 0; k < m; ++k)
    for (int q = 0; q < 3; ++q) {
      lo[q] = fminf(lo[q], bx[k][q]);
      hi[q] = fmaxf(hi[q], bx[k][3 + q]);
    }
  float off[8][3];
  for (int k = 0; k < m; ++k)
    for (int q = 0; q < 3; ++q) off[k][q] = (bx[k][q] + bx[k][3 + q]) - (lo[q] + hi[q]);
  uint32_t out[8];
  for (int sl = 0; sl < 8; ++sl) out[sl] = kNone;
  uint32_t free_slots = 0xFFu, todo = (1u << m) - 1u;
  for (int r = 0; r < m; ++r) {
    float best_sc = -INFINITY;
    int bk = 0, bs = 0;
    for (int k = 0; k < m; ++k) {
      if (!(todo >> k & 1u)) continue;
      for (int sl = 0; sl < 8; ++sl) {
        if (!(free_slots >> sl & 1u)) continue;
        const float sc = ((sl & 1) ? off[k][0] : -off[k][0]) + ((sl & 2) ? off[k][1] : -off[k][1]) +
                         ((sl & 4) ? off[k][2] : -off[k][2]);
        if (sc > best_sc) {
          best_sc = sc;
          bk = k;
          bs = sl;
        }
      }
    }
    out[bs] = c[bk];
    free_slots &= ~(1u << bs);
    todo &= ~(1u << bk);
  }
  uint4* o = reinterpret_cast<uint4*>(cut + 8 * (size_t)b);
  o[0] = make_uint4(out[0], out[1], out[2], out[3]);
  o[1] = make_uint4(out[4], out[5], out[6], out[7]);
}

// members of the cut of binary node b in slot order (kNone: empty slot); a
// one-triangle scene has a root with one leaf member
__device__ __forceinline__ void load_cut(uint32_t n, const uint32_t* __restrict__ cut, uint32_t b, uint32_t out[8]) {
  if (n == 1) {
    out[0] = kLeafBit;
    for (int k = 1; k < 8; ++k) out[k] = kNone;
    return;
  }
  const uint4* p = reinterpret_cast<const uint4*>(cut + 8 * (size_t)b);
  const uint4 a = p[0], c = p[1];
  out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
  out[4] = c.x; out[5] = c.y; out[6] = c.z; out[7] = c.w;
}

// B: wide nodes are numbered top down.  Wide node 0 is the binary root; the
// node that processes wide node w allocates consecutive numbers for the
// internal members of its cut (wctr[1]) and consecutive triangle slots for
// its leaf members (wctr[3]), and publishes each internal member's binary
// node as (epoch << 32 | b) in wsrc.  Threads take wide node numbers from a
// ticket (wctr[0]) and wait (bounded) until their number is published or
// the tree is complete: every node allocated has been processed
// (wctr[2] == wctr[1]).  A thread only waits for a number allocated by a
// thread that already holds an earlier ticket, so the waits always end.
constexpr uint32_t kWideSpinLimit = 1u << 22;
constexpr uint32_t kWideErr = 1u;

__global__ void __launch_bounds__(128) k_wide_alloc(uint32_t n, const uint32_t* __restrict__ cut,
                                                    unsigned long long* __restrict__ wsrc,
                                                    uint4* __restrict__ wrec, uint32_t* __restrict__ wctr,
                                                    uint32_t epoch, uint32_t wcap) {
  while (true) {
    const uint32_t i = atomicAdd(&wctr[0], 1u);
    uint32_t b = 0;
    if (i > 0) {
      // poll the own slot; the shared counters only now and then, so that
      // waiting threads do not crowd the lines the producers update
      uint32_t spins = 0, nap = 32;
      while (true) {
        if (i < wcap) {
          const unsigned long long v = ld_acquire_u64(&wsrc[i]);
          if ((uint32_t)(v >> 32) == epoch) {
            b = (uint32_t)v;
            break;
          }
        }
        if ((spins & 15u) == 15u) {
          const uint32_t done = ld_acquire_u32(&wctr[2]);
          const uint32_t alloc = ld_acquire_u32(&wctr[1]);
          if (i >= alloc && done == alloc) return;   // the tree is complete
          if (ld_acquire_u32(&wctr[4])) return;
        }
        if (++spins > kWideSpinLimit) {
          atomicOr(&wctr[4], kWideErr);
          return;
        }
        __nanosleep(nap);
        if (nap < 256) nap <<= 1;
      }
    }
    uint32_t m[8];
    load_cut(n, cut, b, m);
    uint32_t ni = 0, nl = 0;   // inner members, triangles of the leaf slots
    for (int k = 0; k < 8; ++k) {
      if (member_is_inner(m[k])) ++ni;
      else nl += member_tris(m[k]);
    }
    const uint32_t cb = ni ? atomicAdd(&wctr[1], ni) : 0u;
    const uint32_t tb = nl ? atomicAdd(&wctr[3], nl) : 0u;
    if ((ni && cb + ni > wcap) || tb + nl > n) {
      atomicOr(&wctr[4], kWideErr);
      return;
    }
    uint32_t r = 0;
    for (int k = 0; k < 8; ++k)
      if (member_is_inner(m[k])) st_release_u64(&wsrc[cb + r++], ((unsigned long long)epoch << 32) | m[k]);
    wrec[i] = make_uint4(b, cb, tb, 0u);
    __threadfence();
    atomicAdd(&wctr[2], 1u);
  }
}

// C: quantised boxes and the triangle copies of every wide node.  Per axis
// the node stores an exponent e and an origin P on the grid of s = 2^e with
// |P / s| + 255 <= 2^23; child bounds are P + q s, q in [0, 255], rounded
// outward (q_lo = floor, q_hi = ceil).  Every such bound is a float exactly,
// so the decoded box contains the child's box and the traversal's slab test
// keeps its rounding guarantees.  The node keeps P - 2^23 s, so that the
// bound is the exact fma(float(2^23 + q), s, P - 2^23 s) where the bits of
// float(2^23 + q) are 0x4B000000 | q.
__device__ __forceinline__ int ceil_log2(double x) {   // x > 0
  int ex;
  const double m = frexp(x, &ex);   // x = m 2^ex, m in [0.5, 1)
  return m == 0.5 ? ex - 1 : ex;
}

__global__ void __launch_bounds__(128) k_wide_write(uint32_t n, const uint32_t* __restrict__ cut,
                                                    const uint32_t* __restrict__ child, const float* __restrict__ nbox,
                                                    const float4* __restrict__ tri, const uint4* __restrict__ wrec,
                                                    const uint32_t* __restrict__ wctr, uint32_t wcap,
                                                    float4* __restrict__ wnodes, float4* __restrict__ wtri) {
  if (wctr[4]) return;   // pass B failed: the records are incomplete (traversal is refused)
  const uint32_t count = min(wctr[1], wcap);
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < count; w += gridDim.x * blockDim.x) {
    const uint4 rec = wrec[w];
    uint32_t m[8];
    load_cut(n, cut, rec.x, m);
    float bx[8][6];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    uint32_t valid = 0, imask = 0, counts = 0;
    for (int k = 0; k < 8; ++k) {
      if (m[k] == kNone) continue;
      valid |= 1u << k;
      if (member_is_inner(m[k])) imask |= 1u << k;
      counts |= member_tris(m[k]) << (2 * k);
      for (int q = 0; q < 6; ++q) bx[k][q] = nbox[6 * (size_t)member_box(m[k], n) + q];
      for (int q = 0; q < 3; ++q) {
        lo[q] = fmin(lo[q], (double)bx[k][q]);
        hi[q] = fmax(hi[q], (double)bx[k][3 + q]);
      }
    }
    float pp[3];
    uint32_t eb[3];
    uint32_t qw[6][2] = {{0u, 0u}, {0u, 0u}, {0u, 0u}, {0u, 0u}, {0u, 0u}, {0u, 0u}};   // lo x y z, hi x y z
    const double two23 = 8388608.0;
    for (int a = 0; a < 3; ++a) {
      int e = -126;
      if (hi[a] > lo[a]) e = max(e, ceil_log2((hi[a] - lo[a]) / 255.0));
      const double mag = fmax(fabs(lo[a]), fabs(hi[a]));
      if (mag > 0.0) e = max(e, ceil_log2(mag) - 22);
      double s = 0.0, k0 = 0.0;
      for (int it = 0; it < 64; ++it, ++e) {
        s = ldexp(1.0, e);
        k0 = floor(lo[a] / s);
        if (fabs(k0) + 255.0 <= two23 && (k0 + 255.0) * s >= hi[a]) break;
      }
      pp[a] = (float)((k0 - two23) * s);
      eb[a] = (uint32_t)(e + 127);
      for (int k = 0; k < 8; ++k) {
        uint32_t ql = 255u, qh = 0u;   // empty slot: an inverted box
        if (valid >> k & 1u) {
          ql = (uint32_t)(floor((double)bx[k][a] / s) - k0);
          qh = (uint32_t)(ceil((double)bx[k][3 + a] / s) - k0);
        }
        qw[a][k >> 2] |= ql << (8 * (k & 3));
        qw[3 + a][k >> 2] |= qh << (8 * (k & 3));
      }
    }
    float4* o = wnodes + 5 * (size_t)w;
    o[0] = make_float4(pp[0], pp[1], pp[2], __uint_as_float(eb[0] | (eb[1] << 8) | (eb[2] << 16) | (imask << 24)));
    o[1] = make_float4(__uint_as_float(rec.y), __uint_as_float(rec.z), __uint_as_float(valid),
                       __uint_as_float(counts));
    o[2] = make_float4(__uint_as_float(qw[0][0]), __uint_as_float(qw[0][1]), __uint_as_float(qw[1][0]),
                       __uint_as_float(qw[1][1]));
    o[3] = make_float4(__uint_as_float(qw[2][0]), __uint_as_float(qw[2][1]), __uint_as_float(qw[3][0]),
                       __uint_as_float(qw[3][1]));
    o[4] = make_float4(__uint_as_float(qw[4][0]), __uint_as_float(qw[4][1]), __uint_as_float(qw[5][0]),
                       __uint_as_float(qw[5][1]));
    // the triangles of the leaf slots, slot by slot (a group's in depth-first order)
    uint32_t r = 0;
    for (int k = 0; k < 8; ++k) {
      if (m[k] == kNone || member_is_inner(m[k])) continue;
      uint32_t stack[kGroupMax + 1], sp = 0;
      stack[sp++] = member_is_group(m[k]) ? (m[k] & kGroupNodeMask) : m[k];
      while (sp) {
        const uint32_t x = stack[--sp];
        if (x & kLeafBit) {
          const uint32_t j = x & ~kLeafBit;
          const size_t dst = 3 * (size_t)(rec.z + r++);
          for (int c = 0; c < kTriCopies; ++c) {   // every rotated copy
            const size_t off = (size_t)c * 3 * n;
            wtri[off + dst] = tri[off + 3 * (size_t)j];
            wtri[off + dst + 1] = tri[off + 3 * (size_t)j + 1];
            wtri[off + dst + 2] = tri[off + 3 * (size_t)j + 2];
          }
          wtri[(size_t)kTriCopies * 3 * n + dst / 3] = tri[(size_t)kTriCopies * 3 * n + j];
        } else if (sp + 2 <= kGroupMax + 1) {   // always: a group has at most kGroupMax triangles
          stack[sp++] = __ldg(&child[2 * x + 1]);
          stack[sp++] = __ldg(&child[2 * x]);
        }
      }
    }
  }
}

// Lobe density g(x) of a material on [0, pi/2], up to normalisation: cos^C
// (the S term of Eq. 5; A and B are integrated in closed form), the
// Cook-Torrance lobe, or the user's samples (Sec. III-A)
struct LobeShape {
  uint32_t kind;
  float C;          // Eq. 5
  float kd, m, zw;  // Cook-Torrance: diffuse amount, roughness, integral of D(w/2)
};

__device__ __forceinline__ LobeShape lobe_shape(const rr_material& r, uint32_t kind) {
  LobeShape ls;
  ls.kind = kind;
  ls.C = r.C;
  ls.kd = r.A;
  ls.m = r.B;
  ls.zw = 0.f;
  if (kind == kLobeCookTorrance) {
    const float m = r.B;
    ls.zw = 2.0f * (m * 1.77245385090551603f * erff(1.0f / m) * (1.0f + 0.5f * m * m) - m * m * expf(-1.0f / (m * m))) /
            (kPi * m * m);
  }
  return ls;
}

__device__ __forceinline__ float lobe_value(const LobeShape& ls, float x) {
  if (ls.kind == kLobeCookTorrance) {
    const float t = 0.5f * x, c = cosf(t), tt = tanf(t);
    const float d = expf(-tt * tt / (ls.m * ls.m)) / (kPi * ls.m * ls.m * c * c * c * c);
    return ls.kd * 0.5f * cosf(x) + (1.0f - ls.kd) * d / ls.zw;
  }
  return cospow(x, ls.C);
}

__global__ void k_lut_cells(const rr_material* __restrict__ raw, const uint8_t* __restrict__ kinds, uint32_t nm,
                            const float* __restrict__ samples, float* __restrict__ cells) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nm * (uint32_t)kLutCells) return;
  const uint32_t m = g / kLutCells, j = g % kLutCells;
  const float h = kHalfPi / kLutCells;
  if (kinds[m] == kLobeTable) {   // Simpson: exact for the quadratic through the cell's three samples
    const float* t = samples + (size_t)m * kLobeSamples + 2 * j;
    cells[g] = (t[0] + 4.0f * t[1] + t[2]) * (h / 6.0f);
    return;
  }
  const LobeShape ls = lobe_shape(raw[m], kinds[m]);
  const float a = h * (float)j, mid = a + 0.5f * h, half = 0.5f * h;
  // Gauss-Legendre nodes and weights of order 8 (roots of P8)
  const float xg[4] = {0.18343464249564980f, 0.52553240991632899f, 0.79666647741362674f, 0.96028985649753623f};
  const float wg[4] = {0.36268378337836198f, 0.31370664587788729f, 0.22238103445337447f, 0.10122853629037626f};
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) s += wg[q] * (lobe_value(ls, mid - half * xg[q]) + lobe_value(ls, mid + half * xg[q]));
  cells[g] = s * half;
}

__global__ void k_lut_prefix(const rr_material* __restrict__ raw, const uint8_t* __restrict__ kinds, uint32_t nm,
                             const float* __restrict__ samples, const float* __restrict__ cells,
                             float4* __restrict__ lut, MatDev* __restrict__ mats) {
  const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nm) return;
  const rr_material r = raw[m];
  const uint32_t kind = kinds[m];
  const LobeShape ls = lobe_shape(r, kind);
  const float* tab = samples + (size_t)m * kLobeSamples;
  // the density at node k (the slope of the integral table)
  auto node = [&](int k, float x) { return kind == kLobeTable ? tab[2 * k] : lobe_value(ls, x); };
  const float h = kHalfPi / kLutCells;
  const float* cm = cells + (size_t)m * kLutCells;
  float4* L = lut + (size_t)m * (kLutCells + 1);
  // forward prefix G and backward prefix Gc, both Kahan-compensated
  float sum = 0.f, comp = 0.f;
  L[0] = make_float4(0.f, 0.f, node(0, 0.f), 0.f);
  for (int j = 0; j < kLutCells; ++j) {
    const float y = cm[j] - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
    const float x = (j + 1 == kLutCells) ? kHalfPi : h * (float)(j + 1);
    L[j + 1] = make_float4(sum, 0.f, node(j + 1, x), 0.f);
  }
  float csum = 0.f, ccomp = 0.f;
  for (int j = kLutCells - 1; j >= 0; --j) {
    const float y = cm[j] - ccomp;
    const float t = csum + y;
    ccomp = (t - csum) - y;
    csum = t;
    L[j].y = csum;
  }
  MatDev d;
  d.n = sqrtf(r.eps_r);
  d.tan_d = r.loss_tangent;
  const bool eq5 = kind == kLobeEq5;   // other lobes live entirely in the table
  d.A = eq5 ? r.A : 0.0f;
  d.B = eq5 ? r.B : 0.0f;
  d.S = eq5 ? 1.0f - r.A - r.B : 1.0f;
  d.C = r.C;
  d.invZ = 1.0f / (d.A * kPi + 2.0f * d.B + 2.0f * d.S * sum);
  d.pec = (r.flags & RR_MAT_PERFECT_CONDUCTOR) ? 1u : 0u;
  mats[m] = d;
}

}  // namespace rr

namespace rr_host {

using namespace rr;

#define RR_TRY(x)                        \
  do {                                   \
    cudaError_t e__ = (x);               \
    if (e__ != cudaSuccess) return e__;  \
  } while (0)

cudaError_t build_alloc(rr_scene* s) {
  const size_t T = s->nt, V = s->nv, M = s->nm;
  size_t bytes = 0;
  auto alloc = [&](void** p, size_t n) -> cudaError_t {
    if (n == 0) {
      *p = nullptr;
      return cudaSuccess;
    }
    bytes += n;
    return dev_malloc(p, n);
  };
  s->sort_tiles = (uint32_t)((T + kSortTile - 1) / kSortTile);
  RR_TRY(alloc((void**)&s->d_vtx, V * 3 * sizeof(float)));
  RR_TRY(alloc((void**)&s->d_idx, T * 3 * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_mat_id, T * sizeof(uint16_t)));
  RR_TRY(alloc((void**)&s->d_raw_mats, M * sizeof(rr_material)));
  RR_TRY(alloc((void**)&s->d_mats, M * sizeof(MatDev)));
  RR_TRY(alloc((void**)&s->d_lut, M * (kLutCells + 1) * sizeof(float4)));
  RR_TRY(alloc((void**)&s->d_lut_cells, M * kLutCells * sizeof(float)));
  RR_TRY(alloc((void**)&s->d_lobe_kind, M * sizeof(uint8_t)));
  RR_TRY(alloc((void**)&s->d_tri, (kTriCopies * 3 + 1) * T * sizeof(float4)));
  RR_TRY(alloc((void**)&s->d_nodes, (T > 1 ? T - 1 : 0) * 4 * sizeof(float4)));
  RR_TRY(alloc((void**)&s->d_centroid, T * sizeof(float4)));
  for (int k = 0; k < 2; ++k) {
    RR_TRY(alloc((void**)&s->d_keys[k], T * sizeof(uint32_t)));
    RR_TRY(alloc((void**)&s->d_vals[k], T * sizeof(uint32_t)));
  }
  // the four passes' counters, then the tile sums of the multi-block counter scan
  const size_t hist_words = (size_t)256 * (s->sort_tiles ? s->sort_tiles : 1);
  RR_TRY(alloc((void**)&s->d_hist, (4 * hist_words + scan_tile_words(hist_words)) * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_parent, (T ? 2 * T - 1 : 1) * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_child, (T > 1 ? T - 1 : 1) * 2 * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_nbox, (T ? 2 * T - 1 : 1) * 6 * sizeof(float)));
  RR_TRY(alloc((void**)&s->d_visit, (T > 1 ? T - 1 : 1) * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_misc, 8 * sizeof(uint32_t)));
  RR_TRY(cudaMemset(s->d_misc, 0, 8 * sizeof(uint32_t)));   // status of an empty scene: no error
  RR_TRY(alloc((void**)&s->d_range, (T > 1 ? T - 1 : 1) * sizeof(uint2)));
  // wide BVH: at most T - 1 wide nodes (each owns a distinct binary internal node)
  s->wcap = T > 1 ? (uint32_t)(T - 1) : 1u;
  if (T) {
    RR_TRY(alloc((void**)&s->d_cut, (size_t)s->wcap * 8 * sizeof(uint32_t)));
    RR_TRY(alloc((void**)&s->d_wnodes, (size_t)s->wcap * kWideNodeWords * sizeof(float4)));
    RR_TRY(alloc((void**)&s->d_wtri, (kTriCopies * 3 + 1) * T * sizeof(float4)));
    RR_TRY(alloc((void**)&s->d_wsrc, (size_t)s->wcap * sizeof(unsigned long long)));
    RR_TRY(alloc((void**)&s->d_wrec, (size_t)s->wcap * sizeof(uint4)));
    RR_TRY(alloc((void**)&s->d_wctr, 8 * sizeof(uint32_t)));
    RR_TRY(cudaMemset(s->d_wsrc, 0, (size_t)s->wcap * sizeof(unsigned long long)));   // epoch 0: nothing published
    RR_TRY(cudaMemset(s->d_wctr, 0, 8 * sizeof(uint32_t)));
  }
  s->scene_bytes = bytes;
  return cudaSuccess;
}

cudaError_t build_materials(rr_scene* s, cudaStream_t st) {
  if (s->nm == 0) return cudaSuccess;
  RR_TRY(cudaMemcpyAsync(s->d_lobe_kind, s->lobe_kind.data(), s->nm, cudaMemcpyHostToDevice, st));
  const uint32_t cells = s->nm * kLutCells;
  k_lut_cells<<<(cells + 255) / 256, 256, 0, st>>>(s->d_raw_mats, s->d_lobe_kind, s->nm, s->d_lobe_samples,
                                                     s->d_lut_cells);
  RR_TRY(cudaGetLastError());
  k_lut_prefix<<<(s->nm + 63) / 64, 64, 0, st>>>(s->d_raw_mats, s->d_lobe_kind, s->nm, s->d_lobe_samples,
                                                   s->d_lut_cells, s->d_lut, s->d_mats);
  RR_TRY(cudaGetLastError());
  return cudaStreamSynchronize(st);   // the host copy of the kinds must outlive the upload
}

// buffers of the SAH top, allocated with the first build that uses it
static cudaError_t top_alloc(rr_scene* s) {
  if (s->d_top_ctr) return cudaSuccess;
  const size_t T = s->nt;
  s->cl_blocks = (uint32_t)((T + kClTile - 1) / kClTile);
  const size_t nb4 = (s->cl_blocks + 3u) & ~3u;
  size_t bytes = 0;
  auto alloc = [&](void** p, size_t n) -> cudaError_t {
    bytes += n;
    return dev_malloc(p, n);
  };
  RR_TRY(alloc((void**)&s->d_cl_at, T * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_cl_bsum, nb4 * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_cl_rec, 2 * T * 2 * sizeof(float4)));
  RR_TRY(alloc((void**)&s->d_top_slot, T * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_top_task, T * sizeof(uint4)));
  RR_TRY(alloc((void**)&s->d_top_ready, T * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_top_small, T * sizeof(uint4)));
  RR_TRY(alloc((void**)&s->d_top_ctr, 8 * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_top_cb, T * 6 * sizeof(uint32_t)));
  s->scene_bytes += bytes;
  return cudaSuccess;
}

// a5b on the refitted LBVH (more than kClusterMax triangles)
static cudaError_t build_sah_top(rr_scene* s, cudaStream_t st) {
  const uint32_t n = s->nt;
  RR_TRY(top_alloc(s));
  const uint32_t nb4 = (s->cl_blocks + 3u) & ~3u;
  RR_TRY(cudaMemsetAsync(s->d_cl_at, 0xFF, (size_t)n * sizeof(uint32_t), st));
  RR_TRY(cudaMemsetAsync(s->d_cl_bsum, 0, (size_t)nb4 * sizeof(uint32_t), st));
  RR_TRY(cudaMemsetAsync(s->d_top_ready, 0, (size_t)n * sizeof(uint32_t), st));
  RR_TRY(cudaMemsetAsync(s->d_top_ctr, 0, 8 * sizeof(uint32_t), st));
  k_top_mark<<<(n - 1 + 255) / 256, 256, 0, st>>>(n, s->d_child, s->d_range, s->d_cl_at, s->d_top_slot, s->d_top_ctr,
                                                  s->d_top_cb);
  RR_TRY(cudaGetLastError());
  k_top_count<<<s->cl_blocks, 256, 0, st>>>(n, s->d_cl_at, s->d_cl_bsum);
  RR_TRY(cudaGetLastError());
  k_scan_single<<<1, 1024, 0, st>>>(s->d_cl_bsum, nb4);
  RR_TRY(cudaGetLastError());
  k_top_compact<<<s->cl_blocks, 256, 0, st>>>(n, s->d_cl_at, s->d_cl_bsum, s->d_range, s->d_nbox, s->d_cl_rec,
                                               s->d_top_task, s->d_top_ready, s->d_top_small, s->d_top_ctr,
                                               s->d_top_cb);
  RR_TRY(cudaGetLastError());
  TopArgs a;
  a.rec[0] = s->d_cl_rec;
  a.rec[1] = s->d_cl_rec + 2 * (size_t)n;
  a.slot = s->d_top_slot;
  a.task = s->d_top_task;
  a.ready = s->d_top_ready;
  a.small = s->d_top_small;
  a.ctr = s->d_top_ctr;
  a.cb = s->d_top_cb;
  a.nodes = s->d_nodes;
  a.child = s->d_child;
  a.parent = s->d_parent;
  a.nbox = s->d_nbox;
  a.misc = s->d_misc;
  a.n = n;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  // persistent blocks; a block that finds no task left returns at once
  k_top_sah<<<std::min<uint32_t>((uint32_t)sms * 4u, n / 64u + 1u), kTopBlock, 0, st>>>(a);
  RR_TRY(cudaGetLastError());
  k_top_small<<<std::min<uint32_t>((uint32_t)sms * 4u, n / 256u + 1u), 32 * kSmallWarps, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t build_lbvh(rr_scene* s, cudaStream_t st, bool with_depth) {
  const uint32_t n = s->nt;
  // bounds reset: min slots to all ones, max slots, error and depth to zero
  RR_TRY(cudaMemsetAsync(s->d_misc, 0xFF, 3 * sizeof(uint32_t), st));
  RR_TRY(cudaMemsetAsync(s->d_misc + 3, 0, 5 * sizeof(uint32_t), st));
  if (n == 0) return cudaSuccess;
  const int B = 256;
  const uint32_t g = (n + B - 1) / B;
  const bool sah_top = s->cfg.bvh_build == RR_BVH_SAH_TOP && n > kClusterMax;
  s->launches += ((n > 1) ? (with_depth ? 14u : 13u) : 11u) + (sah_top ? 6u : 0u) +
                 ((size_t)256 * s->sort_tiles > kScanSingleMax ? 8u : 0u);   // 3 launches per pass's counter scan
  k_ingest<<<g, B, 0, st>>>(s->d_vtx, s->d_idx, s->d_mat_id, s->nv, n, s->nm, s->d_centroid, s->d_misc);
  RR_TRY(cudaGetLastError());
  // the four passes' digit counts per tile, zeroed, counted as each pass's input is written
  const size_t hist_words = (size_t)256 * s->sort_tiles;
  RR_TRY(cudaMemsetAsync(s->d_hist, 0, 4 * hist_words * sizeof(uint32_t), st));
  k_morton<<<g, B, 0, st>>>(s->d_centroid, s->d_misc, n, s->d_keys[0], s->d_vals[0], s->sort_tiles, s->d_hist);
  RR_TRY(cudaGetLastError());
  // 30-bit keys: passes over bits 0-7, 8-15, 16-23, 24-29
  int cur = 0;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 8 * pass;
    uint32_t* hist = s->d_hist + pass * hist_words;
    if (hist_words <= kScanSingleMax) {
      k_scan_single<<<1, 1024, 0, st>>>(hist, (uint32_t)hist_words);
    } else {
      uint32_t* tsum = s->d_hist + 4 * hist_words;
      const uint32_t nb = scan_tiles(hist_words), n4 = (uint32_t)(hist_words / 4);
      k_scan_tiles_up<<<nb, kScanBlock, 0, st>>>(hist, n4, tsum, scan_tile_words(hist_words));
      RR_TRY(cudaGetLastError());
      k_scan_single<<<1, 1024, 0, st>>>(tsum, scan_tile_words(hist_words));
      RR_TRY(cudaGetLastError());
      k_scan_tiles_down<<<nb, kScanBlock, 0, st>>>(hist, n4, tsum);
    }
    RR_TRY(cudaGetLastError());
    k_radix_scatter<<<s->sort_tiles, kSortBlock, 0, st>>>(s->d_keys[cur], s->d_vals[cur], s->d_keys[cur ^ 1],
                                                          s->d_vals[cur ^ 1], n, shift, s->sort_tiles, hist,
                                                          pass < 3 ? hist + hist_words : nullptr);
    RR_TRY(cudaGetLastError());
    cur ^= 1;
  }
  // after an even number of passes the sorted pairs are back in slot 0
  k_gather<<<g, B, 0, st>>>(s->d_vtx, s->d_idx, s->d_mat_id, s->d_vals[cur], s->nv, n, s->d_tri, s->d_nbox);
  RR_TRY(cudaGetLastError());
  if (n > 1) {
    k_karras<<<(n - 1 + B - 1) / B, B, 0, st>>>(s->d_keys[cur], (int)n, s->d_child, s->d_parent, s->d_visit,
                                                s->d_range);
    RR_TRY(cudaGetLastError());
    k_refit<<<(n + kRefitBlock - 1) / kRefitBlock, kRefitBlock, 0, st>>>(n, s->d_child, s->d_parent, s->d_range,
                                                                           s->d_visit, s->d_nbox, s->d_nodes);
    RR_TRY(cudaGetLastError());
    if (sah_top) RR_TRY(build_sah_top(s, st));
    if (with_depth) {
      // the stack bound is checked once at creation; on rebuilds the
      // traversal's own stack check reports a deeper tree
      k_depth<<<g, B, 0, st>>>(n, s->d_parent, s->d_misc);
      RR_TRY(cudaGetLastError());
    }
  } else {
    RR_TRY(cudaMemsetAsync(s->d_parent, 0xFF, sizeof(uint32_t), st));
  }
  s->wide_stale = true;   // the 8-wide BVH is collapsed when a scan first needs it
  return cudaSuccess;
}

// a6: the 8-wide quantised BVH, collapsed from the current binary LBVH
cudaError_t build_wide(rr_scene* s, cudaStream_t st) {
  const uint32_t n = s->nt;
  s->wide_stale = false;
  if (n == 0) return cudaSuccess;
  s->launches += 3u;
  s->wide_epoch += 1u;
  if (s->wide_epoch == 0u) s->wide_epoch = 1u;   // 0 marks "never published"
  k_wide_cut<<<n > 1 ? (n - 1 + 127) / 128 : 1, 128, 0, st>>>(n, s->d_child, s->d_nbox, s->d_cut, s->d_wctr);
  RR_TRY(cudaGetLastError());
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t alloc_threads = 2u * 128u * (uint32_t)sms;
  const uint32_t alloc_grid = (std::min<uint32_t>(alloc_threads, s->wcap + 128u) + 127u) / 128u;
  k_wide_alloc<<<alloc_grid, 128, 0, st>>>(n, s->d_cut, s->d_wsrc, s->d_wrec, s->d_wctr, s->wide_epoch, s->wcap);
  RR_TRY(cudaGetLastError());
  k_wide_write<<<std::min<uint32_t>((s->wcap + 127u) / 128u, 8u * (uint32_t)sms), 128, 0, st>>>(
      n, s->d_cut, s->d_child, s->d_nbox, s->d_tri, s->d_wrec, s->d_wctr, s->wcap, s->d_wnodes, s->d_wtri);
  return cudaGetLastError();
}

// Failure detection: the bounded waits of the top build and of the wide
// collapse, each run by its own kernel on counters arranged so that the flag
// it waits for is never set.  `scratch` holds at least 32 zeroed words.
// Returns whether the wait gave up and raised its error bit.
cudaError_t selftest_top_wait(uint32_t* scratch, cudaStream_t st, bool* gave_up) {
  // block task 0 taken and never published, one task pending forever:
  // C = 64 clusters, the marked top part consistent (C - 2 slots after the root)
  uint32_t* ctr = scratch;        // [8]
  uint32_t* ready = scratch + 8;  // [1]
  uint32_t* misc = scratch + 16;  // [8]
  const uint32_t init[8] = {0u, 0u, 62u, 64u, 1u, 1u, 0u, 0u};   // head, slots, marked, clusters, tasks, pending, small, small head
  RR_TRY(cudaMemcpyAsync(ctr, init, sizeof init, cudaMemcpyHostToDevice, st));
  TopArgs a;
  memset(&a, 0, sizeof a);
  a.ready = ready;
  a.ctr = ctr;
  a.misc = misc;
  a.n = 64u;
  k_top_sah<<<1, kTopBlock, 0, st>>>(a);
  RR_TRY(cudaGetLastError());
  uint32_t err = 0;
  RR_TRY(cudaMemcpyAsync(&err, misc + 6, sizeof err, cudaMemcpyDeviceToHost, st));
  RR_TRY(cudaStreamSynchronize(st));
  *gave_up = (err & kErrTopBuild) != 0u;
  return cudaSuccess;
}

cudaError_t selftest_wide_wait(uint32_t* scratch, cudaStream_t st, bool* gave_up) {
  // ticket 1 handed out, wide node 1 allocated but never published (epoch 1)
  uint32_t* wctr = scratch;                                                       // [8]
  unsigned long long* wsrc = reinterpret_cast<unsigned long long*>(scratch + 8);   // [2]
  const uint32_t init[8] = {1u, 2u, 0u, 0u, 0u, 0u, 0u, 0u};   // ticket, allocated, done, triangles, error
  RR_TRY(cudaMemcpyAsync(wctr, init, sizeof init, cudaMemcpyHostToDevice, st));
  k_wide_alloc<<<1, 1, 0, st>>>(1u, nullptr, wsrc, nullptr, wctr, 1u, 2u);
  RR_TRY(cudaGetLastError());
  uint32_t err = 0;
  RR_TRY(cudaMemcpyAsync(&err, wctr + 4, sizeof err, cudaMemcpyDeviceToHost, st));
  RR_TRY(cudaStreamSynchronize(st));
  *gave_up = (err & kWideErr) != 0u;
  return cudaSuccess;
}

}  // namespace rr_host
