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
__global__ void k_morton(const float4* __restrict__ centroid, const uint32_t* __restrict__ misc, uint32_t nt,
                         uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
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
  keys[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
  vals[i] = i;
}

// ---------------------------------------------------------------------------
// a3: LSD radix sort, 8-bit digits.  hist is digit major: hist[d * tiles + t].
__global__ void k_radix_hist(const uint32_t* __restrict__ keys, uint32_t n, int shift, uint32_t tiles,
                             uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t base = blockIdx.x * kSortTile;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const uint32_t i = base + r * kSortBlock + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of n counters (n a multiple of 4, 16-byte aligned) with one
// block: chunks of blockDim x 4 counters, one coalesced uint4 per thread,
// carried from chunk to chunk
__global__ void k_scan_single(uint32_t* __restrict__ data, uint32_t n) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  const uint32_t t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  if (t == 0) s_carry = 0u;
  __syncthreads();
  uint4* d4 = reinterpret_cast<uint4*>(data);
  const uint32_t n4 = n / 4u;
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

// stable scatter: keys of a tile are ranked in index order (round, warp, lane)
__global__ void k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, uint32_t n, int shift,
                                uint32_t tiles, const uint32_t* __restrict__ offs) {
  __shared__ uint32_t s_base[256];
  __shared__ uint32_t s_warp[kSortBlock / 32][256];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  s_base[t] = offs[t * tiles + blockIdx.x];
  const uint32_t base = blockIdx.x * kSortTile;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < kSortItems; ++r) {
    for (int w = 0; w < kSortBlock / 32; ++w) s_warp[w][t] = 0;
    __syncthreads();
    const uint32_t i = base + r * kSortBlock + t;
    const bool valid = i < n;
    const uint32_t key = valid ? kin[i] : 0u;
    const uint32_t digit = (key >> shift) & 255u;
    const uint32_t tag = valid ? digit : 256u + (uint32_t)lane;   // invalid lanes match only themselves
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, tag);
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
      vout[pos] = vin[i];
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
  tri[3 * j + 0] = make_float4(v[0].x, v[0].y, v[0].z, __uint_as_float(t));
  tri[3 * j + 1] = make_float4(v[1].x, v[1].y, v[1].z, __uint_as_float((uint32_t)mat_id[t]));
  tri[3 * j + 2] = make_float4(v[2].x, v[2].y, v[2].z, 0.0f);
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
                         uint32_t* __restrict__ parent, uint32_t* __restrict__ visit) {
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
  parent[(left & kLeafBit) ? (n - 1 + (left & ~kLeafBit)) : left] = (uint32_t)i;
  parent[(right & kLeafBit) ? (n - 1 + (right & ~kLeafBit)) : right] = (uint32_t)i;
  visit[i] = 0;
  if (i == 0) parent[0] = kNone;
}

__device__ __forceinline__ uint32_t node_slot(uint32_t c, uint32_t n) {
  return (c & kLeafBit) ? (n - 1 + (c & ~kLeafBit)) : c;
}

// a5: each leaf walks to the root; at every internal node the first arrival
// stops and the second merges both child boxes (they are final by then)
__global__ void k_refit(uint32_t n, const uint32_t* __restrict__ child, const uint32_t* __restrict__ parent,
                        uint32_t* __restrict__ visit, float* __restrict__ nbox, float4* __restrict__ nodes) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  uint32_t p = parent[n - 1 + j];
  while (p != kNone) {
    // acquire-release: the second arrival sees the first one's box
    cuda::atomic_ref<uint32_t, cuda::thread_scope_device> cnt(visit[p]);
    if (cnt.fetch_add(1u, cuda::memory_order_acq_rel) == 0u) return;
    const uint32_t c0 = child[2 * p], c1 = child[2 * p + 1];
    const float* b0p = nbox + 6 * (size_t)node_slot(c0, n);
    const float* b1p = nbox + 6 * (size_t)node_slot(c1, n);
    float b0[6], b1[6];
    for (int k = 0; k < 6; ++k) {
      b0[k] = __ldcg(b0p + k);
      b1[k] = __ldcg(b1p + k);
    }
    float4* nd = nodes + 4 * (size_t)p;
    nd[0] = make_float4(b0[0], b0[3], b0[1], b0[4]);
    nd[1] = make_float4(b1[0], b1[3], b1[1], b1[4]);
    nd[2] = make_float4(b0[2], b0[5], b1[2], b1[5]);
    nd[3] = make_float4(__uint_as_float(c0), __uint_as_float(c1), 0.f, 0.f);
    float* bp = nbox + 6 * (size_t)p;
    for (int k = 0; k < 3; ++k) {
      __stcg(bp + k, fminf(b0[k], b1[k]));
      __stcg(bp + 3 + k, fmaxf(b0[3 + k], b1[3 + k]));
    }
    p = parent[p];
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
  c[0] = __ldg(&child[2 * b]);
  c[1] = __ldg(&child[2 * b + 1]);
  int m = 2;
  for (int k = 0; k < 2; ++k)
    for (int q = 0; q < 6; ++q) bx[k][q] = __ldg(&nbox[6 * (size_t)node_slot(c[k], n) + q]);
  while (m < 8) {
    int best = -1;
    float best_a = -1.0f;
    for (int k = 0; k < m; ++k) {
      if (c[k] & kLeafBit) continue;
      const float a = box_area(bx[k]);
      if (a > best_a) {
        best_a = a;
        best = k;
      }
    }
    if (best < 0) break;
    const uint32_t p = c[best];
    const uint32_t c0 = __ldg(&child[2 * p]), c1 = __ldg(&child[2 * p + 1]);
    c[best] = c0;
    c[m] = c1;
    for (int q = 0; q < 6; ++q) {
      bx[best][q] = __ldg(&nbox[6 * (size_t)node_slot(c0, n) + q]);
      bx[m][q] = __ldg(&nbox[6 * (size_t)node_slot(c1, n) + q]);
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
    uint32_t ni = 0, nl = 0;
    for (int k = 0; k < 8; ++k) {
      if (m[k] == kNone) continue;
      if (m[k] & kLeafBit) ++nl;
      else ++ni;
    }
    const uint32_t cb = ni ? atomicAdd(&wctr[1], ni) : 0u;
    const uint32_t tb = nl ? atomicAdd(&wctr[3], nl) : 0u;
    if ((ni && cb + ni > wcap) || tb + nl > n) {
      atomicOr(&wctr[4], kWideErr);
      return;
    }
    uint32_t r = 0;
    for (int k = 0; k < 8; ++k)
      if (m[k] != kNone && !(m[k] & kLeafBit))
        st_release_u64(&wsrc[cb + r++], ((unsigned long long)epoch << 32) | m[k]);
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
                                                    const float* __restrict__ nbox,
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
    uint32_t valid = 0, imask = 0;
    for (int k = 0; k < 8; ++k) {
      if (m[k] == kNone) continue;
      valid |= 1u << k;
      if (!(m[k] & kLeafBit)) imask |= 1u << k;
      for (int q = 0; q < 6; ++q) bx[k][q] = nbox[6 * (size_t)node_slot(m[k], n) + q];
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
    o[1] = make_float4(__uint_as_float(rec.y), __uint_as_float(rec.z), __uint_as_float(valid), 0.0f);
    o[2] = make_float4(__uint_as_float(qw[0][0]), __uint_as_float(qw[0][1]), __uint_as_float(qw[1][0]),
                       __uint_as_float(qw[1][1]));
    o[3] = make_float4(__uint_as_float(qw[2][0]), __uint_as_float(qw[2][1]), __uint_as_float(qw[3][0]),
                       __uint_as_float(qw[3][1]));
    o[4] = make_float4(__uint_as_float(qw[4][0]), __uint_as_float(qw[4][1]), __uint_as_float(qw[5][0]),
                       __uint_as_float(qw[5][1]));
    uint32_t r = 0;
    for (int k = 0; k < 8; ++k) {
      if (m[k] == kNone || !(m[k] & kLeafBit)) continue;
      const uint32_t j = m[k] & ~kLeafBit;
      const size_t dst = 3 * (size_t)(rec.z + r++);
      wtri[dst] = tri[3 * (size_t)j];
      wtri[dst + 1] = tri[3 * (size_t)j + 1];
      wtri[dst + 2] = tri[3 * (size_t)j + 2];
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
    return cudaMalloc(p, n);
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
  RR_TRY(alloc((void**)&s->d_tri, T * 3 * sizeof(float4)));
  RR_TRY(alloc((void**)&s->d_nodes, (T > 1 ? T - 1 : 0) * 4 * sizeof(float4)));
  RR_TRY(alloc((void**)&s->d_centroid, T * sizeof(float4)));
  for (int k = 0; k < 2; ++k) {
    RR_TRY(alloc((void**)&s->d_keys[k], T * sizeof(uint32_t)));
    RR_TRY(alloc((void**)&s->d_vals[k], T * sizeof(uint32_t)));
  }
  RR_TRY(alloc((void**)&s->d_hist, (size_t)256 * (s->sort_tiles ? s->sort_tiles : 1) * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_parent, (T ? 2 * T - 1 : 1) * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_child, (T > 1 ? T - 1 : 1) * 2 * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_nbox, (T ? 2 * T - 1 : 1) * 6 * sizeof(float)));
  RR_TRY(alloc((void**)&s->d_visit, (T > 1 ? T - 1 : 1) * sizeof(uint32_t)));
  RR_TRY(alloc((void**)&s->d_misc, 8 * sizeof(uint32_t)));
  // wide BVH: at most T - 1 wide nodes (each owns a distinct binary internal node)
  s->wcap = T > 1 ? (uint32_t)(T - 1) : 1u;
  if (T) {
    RR_TRY(alloc((void**)&s->d_cut, (size_t)s->wcap * 8 * sizeof(uint32_t)));
    RR_TRY(alloc((void**)&s->d_wnodes, (size_t)s->wcap * kWideNodeWords * sizeof(float4)));
    RR_TRY(alloc((void**)&s->d_wtri, T * 3 * sizeof(float4)));
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

cudaError_t build_lbvh(rr_scene* s, cudaStream_t st, bool with_depth) {
  const uint32_t n = s->nt;
  if (n == 0) return cudaSuccess;
  // bounds reset: min slots to all ones, max slots, error and depth to zero
  RR_TRY(cudaMemsetAsync(s->d_misc, 0xFF, 3 * sizeof(uint32_t), st));
  RR_TRY(cudaMemsetAsync(s->d_misc + 3, 0, 5 * sizeof(uint32_t), st));
  const int B = 256;
  const uint32_t g = (n + B - 1) / B;
  s->launches += (n > 1) ? (with_depth ? 18u : 17u) : 15u;
  k_ingest<<<g, B, 0, st>>>(s->d_vtx, s->d_idx, s->d_mat_id, s->nv, n, s->nm, s->d_centroid, s->d_misc);
  RR_TRY(cudaGetLastError());
  k_morton<<<g, B, 0, st>>>(s->d_centroid, s->d_misc, n, s->d_keys[0], s->d_vals[0]);
  RR_TRY(cudaGetLastError());
  // 30-bit keys: passes over bits 0-7, 8-15, 16-23, 24-29
  int cur = 0;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 8 * pass;
    k_radix_hist<<<s->sort_tiles, kSortBlock, 0, st>>>(s->d_keys[cur], n, shift, s->sort_tiles, s->d_hist);
    RR_TRY(cudaGetLastError());
    k_scan_single<<<1, 1024, 0, st>>>(s->d_hist, 256u * s->sort_tiles);
    RR_TRY(cudaGetLastError());
    k_radix_scatter<<<s->sort_tiles, kSortBlock, 0, st>>>(s->d_keys[cur], s->d_vals[cur], s->d_keys[cur ^ 1],
                                                          s->d_vals[cur ^ 1], n, shift, s->sort_tiles, s->d_hist);
    RR_TRY(cudaGetLastError());
    cur ^= 1;
  }
  // after an even number of passes the sorted pairs are back in slot 0
  k_gather<<<g, B, 0, st>>>(s->d_vtx, s->d_idx, s->d_mat_id, s->d_vals[cur], s->nv, n, s->d_tri, s->d_nbox);
  RR_TRY(cudaGetLastError());
  if (n > 1) {
    k_karras<<<(n - 1 + B - 1) / B, B, 0, st>>>(s->d_keys[cur], (int)n, s->d_child, s->d_parent, s->d_visit);
    RR_TRY(cudaGetLastError());
    k_refit<<<g, B, 0, st>>>(n, s->d_child, s->d_parent, s->d_visit, s->d_nbox, s->d_nodes);
    RR_TRY(cudaGetLastError());
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
      n, s->d_cut, s->d_nbox, s->d_tri, s->d_wrec, s->d_wctr, s->wcap, s->d_wnodes, s->d_wtri);
  return cudaGetLastError();
}

}  // namespace rr_host
