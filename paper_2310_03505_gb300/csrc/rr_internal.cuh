// rr_internal.cuh -- device layouts and helpers shared by the CUDA
// translation units of the radar scan library (never by the oracle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rr.h"

namespace rr {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kAir = 0xFFFFu;
constexpr uint32_t kLeafBit = 0x80000000u;
constexpr int kStack = 64;            // traversal stack entries; the build checks depth <= kStack
constexpr int kLutCells = 2048;       // lobe table cells over [0, pi/2]
constexpr int kLobeSamples = 2 * kLutCells + 1;   // samples of a tabulated lobe (RR_LOBE_SAMPLES)
constexpr uint32_t kLobeEq5 = 0, kLobeCookTorrance = 1, kLobeTable = 2;
constexpr float kPi = 3.14159265358979323846f;
constexpr float kHalfPi = 1.57079632679489661923f;
constexpr float kC0 = 299792458.0f;   // speed of light (m/s)
constexpr uint32_t kSpinLimit = 1u << 21;  // bounded device waits (each spin re-reads a flag from L2: about a second)

// status bits of the sticky device error word
constexpr uint32_t kErrCapacityRays = 1u;
constexpr uint32_t kErrCapacityRecs = 2u;
constexpr uint32_t kErrTimeout = 4u;
constexpr uint32_t kErrCapacitySegs = 8u;
constexpr uint32_t kErrBadVertex = 16u;
constexpr uint32_t kErrStack = 32u;
constexpr uint32_t kErrBvh = 64u;      // the BVH build failed (traversal refused)
constexpr uint32_t kErrTopBuild = 0x100u;   // build status word: the SAH top build was abandoned

// ---------------------------------------------------------------------------
// device material record (derived at scene creation)
struct __align__(16) MatDev {
  float n;          // refractive index sqrt(eps_r)
  float tan_d;      // loss tangent
  float A, B;       // Eq. 5
  float S, C;       // S = 1 - A - B
  float invZ;       // 1 / (A pi + 2 B + 2 S G(pi/2)), G from the lobe table
  uint32_t pec;     // perfect conductor
};

// Triangle vertices are stored three times, with their coordinates rotated
// by 0, 1 and 2 places: copy r holds (v[k], v[k+1 mod 3], v[k+2 mod 3]) for
// k = r.  The watertight ray/triangle test works in a frame whose third axis
// is the ray's dominant axis kz and whose first two axes follow it cyclically;
// that frame is copy r = (kz + 1) mod 3, so the test reads the vertices in its
// own order instead of selecting each coordinate at run time.
constexpr int kTriCopies = 3;
__device__ __forceinline__ float3 tri_rotate(float3 v, uint32_t r) {
  return r == 0 ? v : (r == 1 ? make_float3(v.y, v.z, v.x) : make_float3(v.z, v.x, v.y));
}

// ray record, 48 bytes
struct __align__(16) RayRec {
  float4 o_L;   // origin, one-way optical path so far
  float4 d_E;   // unit direction, energy
  uint4 meta;   // x: prev leaf (sorted index) or kNone, y: az << 16 | k,
                // z: path (bit 31: masked), w: scan << 16 | (medium material or kAir)
};

// An air-path candidate whose visibility is still open (Sec. III-A): what the
// visibility query needs and what it changes once the sensor is visible.  It
// is written over the candidate's ray record of the bounce, which the shading
// pass has consumed (48 bytes, the size of a RayRec).
struct __align__(16) VisJob {
  float4 p_leaf;   // hit point, the hit leaf (bits): the query starts there
  uint4 idx;       // scan; queue position of the child the air-path return depletes (kNone: not spawned);
                   // position of its reserved return record (kNone: none); tally slot (kNone: no tallies)
  float4 val;      // x: the child energy before the return is taken, y: the return, z: its image energy
                   // (speckle and range weight applied), w: segment slot (bits; kNone: no dump)
};

static_assert(sizeof(VisJob) == sizeof(RayRec), "a VisJob takes the place of a RayRec");

// hit record, 16 bytes
struct __align__(16) HitRec {
  float t;
  uint32_t leaf;   // sorted leaf index or kNone
  uint32_t flags;  // bit 0: visibility test ran, bit 1: visible
  float wa_g;      // W(omega_a) of a visible air-path candidate, else 0 (the receive weight is applied by the shading)
};

// device counters of one scene
struct ScanCounters {
  uint32_t count[RR_MAX_BOUNCES + 1];      // queue length per bounce
  uint32_t rec_start[RR_MAX_BOUNCES + 1];  // first record of each bounce
  uint32_t seg_start[RR_MAX_BOUNCES + 1];  // first debug segment of each bounce
  uint32_t trace_ticket[RR_MAX_BOUNCES];
  uint32_t shade_ticket[RR_MAX_BOUNCES];
  uint32_t vis_count[RR_MAX_BOUNCES];      // visibility jobs per bounce
  uint32_t vis_ticket[RR_MAX_BOUNCES];
  uint32_t need_rays, need_recs;           // largest request seen (overflow report)
  uint32_t error;                          // sticky kErr* bits
  uint32_t pad;
  unsigned long long stat_closest, stat_anyhit, stat_returns, stat_scans;
  unsigned long long stat_nodes, stat_tris;
  unsigned long long stat_nodes_any, stat_tris_any;
};

// 8-wide BVH node with 8-bit quantised child boxes, 5 float4 (80 bytes):
//   w0 = (P.x, P.y, P.z, ex | ey << 8 | ez << 16 | imask << 24)
//   w1 = (first internal child, first triangle, valid mask, leaf counts: 2 bits per slot)
//   w2 = (qlo.x[0..3], qlo.x[4..7], qlo.y[0..3], qlo.y[4..7])       (bytes)
//   w3 = (qlo.z[0..3], qlo.z[4..7], qhi.x[0..3], qhi.x[4..7])
//   w4 = (qhi.y[0..3], qhi.y[4..7], qhi.z[0..3], qhi.z[4..7])
// Slot k of an axis has bounds fma(float(2^23 + q), s, P) with s = 2^(e - 127)
// (exact floats that contain the child's box).  Internal children are stored
// consecutively from the first child in slot order, the triangles of the
// leaf slots (1..3 each, a small binary subtree) likewise from the first
// triangle.
constexpr int kWideNodeWords = 5;

// Return record key: global image column (scan's first column + azimuth)
// and range bin.  Records of one bounce are in column order.
constexpr int kBinBits = 14;                       // n_bins <= RR_MAX_BINS = 2^14
constexpr uint32_t kBinMask = (1u << kBinBits) - 1u;
constexpr uint32_t kMaxColumns = 1u << (32 - kBinBits);   // columns of one launch sequence
constexpr uint32_t kMaxBatchScans = 0xFFFFu;       // scan index lives in 16 bits of RayRec.meta.w
constexpr uint32_t kMediumMask = 0xFFFFu;

// Buckets of the closest-hit query order: direction octant (3 bits), height
// cell (2 bits) and an 8 x 8 grid of horizontal cells (6 bits, Morton order)
// around the scan's sensor
constexpr uint32_t kOrderBuckets = 1u << 11;

// Per-scan constants of a batch (one pose and sensor model), 160 bytes.
// Kernels read the fields of the scan each ray belongs to.
struct __align__(16) ScanDesc {
  float4 pos_rmax;   // sensor position, r_max = n_bins * bin_size
  float4 quat;       // normalised (w, x, y, z), sensor to world
  uint4 dims;        // n_az, ns, max_bounces, n_bins
  float4 beam;       // beam_width b, beam_prob P, elevation, bin_size
  float4 phys;       // t_min, min_energy, freq, r_lim (range limit of a closest-hit query)
  float4 post;       // blur_sigma, az_sigma, noise_sys, noise_amb
  uint4 rng;         // seed_lo, seed_hi, scan_id, flags
  uint4 offs;        // first initial ray, first column, first float of image_tmp (or kNone), first azimuth
  float4 ext;        // beam aspect (elliptic beams), Perlin cell in beams, Perlin cell in bins, range falloff k
  float* image;      // [n_az][n_bins] output (device)
  unsigned long long pad;
};

// Launch-sequence constants of one batch (passed by value)
struct ScanArgs {
  // scene
  const float4* tri;         // [3][T][3] sorted: v0 (w: orig id bits), v1 (w: material bits), v2; copy r holds
                             // the coordinates rotated by r (tri_rotate), so copy 0 is (x, y, z); then [T]
                             // (unit geometric normal, material bits) at tri + 3 tri_copy
  size_t tri_copy;           // float4s from one rotated copy to the next (3 T)
  const float4* nodes;       // [T-1][4] Aila-Laine layout
  const MatDev* mats;
  const float4* lut;         // [M][kLutCells + 1]: (G(x_k), Gc(x_k), cos^C(x_k), 0)
  uint32_t n_tris, n_mats;
  uint32_t wide;             // nodes are 8-wide quantised (tri in wide-leaf order), else binary
  uint32_t node_cap;         // nodes in the node array (traversal bound)
  const uint32_t* bvh_status;   // non-zero: the last build failed, nothing may be traced
  const uint32_t* build_status; // the scene's build status word (kErrTopBuild: nothing may be traced)
  // batch
  const ScanDesc* desc;      // [n_scans]
  const uint32_t* ray0;      // [n_scans + 1] prefix of n_az * ns
  const uint32_t* col0;      // [n_scans + 1] prefix of n_az
  uint32_t n_scans, n_rays0, n_cols;
  uint32_t max_bounces;      // over the batch
  uint32_t max_bins;         // over the batch
  uint32_t any_flags;        // union of the scans' flags
  uint32_t refill;           // a warp hands out new queries once this many lanes are idle (1..32)
  // workspace
  RayRec* rays[2];
  HitRec* hits;
  uint2* recs;               // (column << kBinBits | bin, energy bits)
  unsigned long long* tile_status;
  ScanCounters* ctr;
  float* image_tmp;          // images before the azimuth pattern (or null)
  uint32_t ray_cap, rec_cap;
  // query order of the closest-hit queries of bounces >= 1 (null: queue order)
  uint16_t* order_key;       // [ray_cap] bucket of every queued ray (written by the shading pass)
  uint32_t* order_perm;      // [ray_cap] queue index of the j-th query
  uint32_t* order_hist;      // [RR_MAX_BOUNCES + 1][kOrderBuckets] rays per bucket
  uint32_t* order_off;       // [kOrderBuckets] next free position of every bucket
  // deferred visibility (defer_vis != 0): the shading pass lists the air-path
  // candidates of its bounce (queue indices in vis_list, a VisJob written over
  // each candidate's spent ray record) and the visibility query settles them
  uint32_t defer_vis;
  uint32_t* vis_list;        // [ray_cap]
  // debug (may be null)
  rr_segment* segs;
  uint32_t seg_cap;
  float* tallies;            // [n_rays0][4]
  const uint8_t* mask;       // [n_rays0]
};

// scan and medium of a queued ray; a slot left stale by a failed step (the
// scan then reports an error) still maps to valid table entries
__device__ __forceinline__ uint2 ray_scan_medium(const ScanArgs& a, uint32_t w) {
  uint32_t scan = w >> 16, medium = w & kMediumMask;
  if (scan >= a.n_scans) scan = 0;
  if (medium != kAir && medium >= a.n_mats) medium = kAir;
  return make_uint2(scan, medium);
}

// index of the scan owning item i of a prefix array p[0..n] (p[0] = 0,
// non-decreasing, i < p[n]): the last s with p[s] <= i
__device__ __forceinline__ uint32_t owner_of(const uint32_t* __restrict__ p, uint32_t n, uint32_t i) {
  uint32_t lo = 0, hi = n;   // invariant: p[lo] <= i < p[hi]
  while (hi - lo > 1u) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(&p[mid]) <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC 2011): counter (scan, a, b, c), key = seed
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// uniform in (0,1) from the top 23 bits, (2 (x >> 9) + 1) / 2^24: exact in float
__device__ __forceinline__ float u01(uint32_t x) { return (float)(2u * (x >> 9) + 1u) * 5.9604644775390625e-8f; }

// draw of a scan whose rng words are (seed_lo, seed_hi, scan_id, flags)
__device__ __forceinline__ uint4 draw(uint4 rng, uint32_t w1, uint32_t w2, uint32_t w3) {
  return philox(make_uint4(rng.z, w1, w2, w3), make_uint2(rng.x, rng.y));
}

// ---------------------------------------------------------------------------
// small vector helpers
__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return make_float3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float length(float3 a) { return sqrtf(dot(a, a)); }
// a / |a| with correctly rounded square root and divisions: no systematic
// bias (an approximate reciprocal square root has one, and a ray reflected
// many times between parallel walls accumulates it into its direction)
__device__ __forceinline__ float3 normalize(float3 a) {
  const float n = sqrtf(dot(a, a));
  return make_float3(__fdiv_rn(a.x, n), __fdiv_rn(a.y, n), __fdiv_rn(a.z, n));
}
// angle between two vectors, well conditioned at 0 and pi
__device__ __forceinline__ float angle_between(float3 a, float3 b) { return atan2f(length(cross(a, b)), dot(a, b)); }

// rotate v by the unit quaternion q = (w, x, y, z)
__device__ __forceinline__ float3 qrot(float4 q, float3 v) {
  const float w = q.x, x = q.y, y = q.z, z = q.w;
  return make_float3((1.f - 2.f * (y * y + z * z)) * v.x + 2.f * (x * y - w * z) * v.y + 2.f * (x * z + w * y) * v.z,
                     2.f * (x * y + w * z) * v.x + (1.f - 2.f * (x * x + z * z)) * v.y + 2.f * (y * z - w * x) * v.z,
                     2.f * (x * z - w * y) * v.x + 2.f * (y * z + w * x) * v.y + (1.f - 2.f * (x * x + y * y)) * v.z);
}

// cos^C(x) for x in [0, pi/2] as exp(C log1p(-2 sin^2(x/2))): keeps the
// relative error near 1 ulp for the sharp lobes (C up to a few thousand)
__device__ __forceinline__ float cospow(float x, float C) {
  if (C == 0.0f) return 1.0f;
  const float s = sinf(0.5f * x);
  // at x = pi/2 (rounded up in float) -2 s^2 can land just below -1: clamp so
  // that cos^C(pi/2) = exp(-inf) = 0 instead of NaN
  return expf(C * log1pf(fmaxf(-2.0f * s * s, -1.0f)));
}

// Lobe table of one material: node k at x_k = k (pi/2) / kLutCells holds
// (G(x_k), Gc(x_k), cos^C(x_k), 0) with G(x) = integral of cos^C over [0, x]
// and Gc(x) = integral over [x, pi/2].  Values between nodes come from cubic
// Hermite interpolation (G' = cos^C, Gc' = -cos^C).
__device__ __forceinline__ float lut_interp(const float4* __restrict__ lut, float x, bool comp) {
  const float h = kHalfPi / kLutCells;
  const float u = x * (kLutCells / kHalfPi);
  if (!(u > 0.0f)) return comp ? __ldg(&lut[0]).y : 0.0f;        // also NaN
  if (u >= (float)kLutCells) return comp ? 0.0f : __ldg(&lut[kLutCells]).x;
  const int k = (int)u;
  const float s = u - (float)k;
  const float4 p0 = __ldg(&lut[k]), p1 = __ldg(&lut[k + 1]);
  const float s2 = s * s, s3 = s2 * s;
  const float h00 = 2.f * s3 - 3.f * s2 + 1.f, h10 = s3 - 2.f * s2 + s, h01 = -2.f * s3 + 3.f * s2,
              h11 = s3 - s2;
  if (comp) return h00 * p0.y - h10 * h * p0.z + h01 * p1.y - h11 * h * p1.z;
  return h00 * p0.x + h10 * h * p0.z + h01 * p1.x + h11 * h * p1.z;
}

// integral of cos^C over [lo, hi], -pi/2 <= lo < hi <= pi/2; tails use the
// complementary table so that no large nearly-equal values are subtracted
__device__ __forceinline__ float lut_integral(const float4* __restrict__ lut, float lo, float hi) {
  if (lo >= 0.0f) {
    const float half = 0.5f * __ldg(&lut[kLutCells]).x;
    const float g_lo = lut_interp(lut, lo, false);
    if (g_lo > half) return lut_interp(lut, lo, true) - lut_interp(lut, hi, true);
    return lut_interp(lut, hi, false) - g_lo;
  }
  if (hi <= 0.0f) return lut_integral(lut, -hi, -lo);
  return lut_interp(lut, hi, false) + lut_interp(lut, -lo, false);
}

// Eq. 4 with the normalised Eq. 5 lobe: fraction of the lobe inside the
// window [w - b/2, w + b/2] clipped to [-pi/2, pi/2]
__device__ __forceinline__ float brdf_window(const MatDev& m, const float4* __restrict__ lut, float w, float b) {
  const float lo = fmaxf(w - 0.5f * b, -kHalfPi), hi = fminf(w + 0.5f * b, kHalfPi);
  if (!(hi > lo)) return 0.0f;
  float v = m.A * (hi - lo) + m.B * 2.0f * cosf(0.5f * (hi + lo)) * sinf(0.5f * (hi - lo));
  if (m.S != 0.0f) v += m.S * lut_integral(lut, lo, hi);
  return fmaxf(v * m.invZ, 0.0f);
}

}  // namespace rr
