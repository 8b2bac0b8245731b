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
__global__ void k_lut_cells(const rr_material* __restrict__ raw, uint32_t nm, float* __restrict__ cells) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nm * (uint32_t)kLutCells) return;
  const uint32_t m = g / kLutCells, j = g % kLutCells;
  const float C = raw[m].C;
  const float h = kHalfPi / kLutCells;
  const float a = h * (float)j, mid = a + 0.5f * h, half = 0.5f * h;
  // Gauss-Legendre nodes and weights of order 8 (roots of P8)
  const float xg[4] = {0.18343464249564980f, 0.52553240991632899f, 0.79666647741362674f, 0.96028985649753623f};
  const float wg[4] = {0.36268378337836198f, 0.31370664587788729f, 0.22238103445337447f, 0.10122853629037626f};
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) s += wg[q] * (cospow(mid - half * xg[q], C) + cospow(mid + half * xg[q], C));
  cells[g] = s * half;
}

__global__ void k_lut_prefix(const rr_material* __restrict__ raw, uint32_t nm, const float* __restrict__ cells,
                             float4* __restrict__ lut, MatDev* __restrict__ mats) {
  const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nm) return;
  const rr_material r = raw[m];
  const float h = kHalfPi / kLutCells;
  const float* cm = cells + (size_t)m * kLutCells;
  float4* L = lut + (size_t)m * (kLutCells + 1);
  // forward prefix G and backward prefix Gc, both Kahan-compensated
  float sum = 0.f, comp = 0.f;
  L[0] = make_float4(0.f, 0.f, cospow(0.f, r.C), 0.f);
  for (int j = 0; j < kLutCells; ++j) {
    const float y = cm[j] - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
    const float x = (j + 1 == kLutCells) ? kHalfPi : h * (float)(j + 1);
    L[j + 1] = make_float4(sum, 0.f, cospow(x, r.C), 0.f);
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
  d.A = r.A;
  d.B = r.B;
  d.S = 1.0f - r.A - r.B;
  d.C = r.C;
  d.invZ = 1.0f / (r.A * kPi + 2.0f * r.B + 2.0f * d.S * sum);
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
  s->scene_bytes = bytes;
  return cudaSuccess;
}

cudaError_t build_materials(rr_scene* s, cudaStream_t st) {
  if (s->nm == 0) return cudaSuccess;
  const uint32_t cells = s->nm * kLutCells;
  k_lut_cells<<<(cells + 255) / 256, 256, 0, st>>>(s->d_raw_mats, s->nm, s->d_lut_cells);
  RR_TRY(cudaGetLastError());
  k_lut_prefix<<<(s->nm + 63) / 64, 64, 0, st>>>(s->d_raw_mats, s->nm, s->d_lut_cells, s->d_lut, s->d_mats);
  return cudaGetLastError();
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
  return cudaSuccess;
}

}  // namespace rr_host
