// rr_trace.cu -- wavefront ray tracing of a batch of polar scans.
//
// Per batch: raygen -> { trace -> shade } x max_bounces -> image
// A batch is one or more scans of the same scene, each with its own pose and
// sensor model (ScanDesc); every ray carries the index of its scan, so scans
// of uneven ray counts and bounce limits share every launch.
//   raygen  Sec. III-A, Eq. 2: N_s rays per azimuth beam from the D3 cone.
//   trace   closest hit through the LBVH (watertight ray/triangle test of
//           Woop, Benthin, Wald, JCGT 2013) and, for multipath, the
//           visibility test of the air-path return toward the sensor.
//   shade   Sec. III-A: Fresnel split E0 = E1 + E2, Snell refraction,
//           attenuation in lossy media, traveled-path and air-path returns
//           through the beam window of the material lobe (Eq. 3-5), and the
//           reflected / refracted children.  Children and return records are
//           compacted stably (single pass, decoupled look-back over tiles of
//           256 rays), so every queue and every bounce's record list stays
//           in (azimuth, ray) order.
//
// All kernels are persistent: the grid is a multiple of the SM count and
// reads the queue length from device memory, so a whole batch is a fixed
// sequence of launches with no host round trip between bounces.
#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "rr_host.h"

namespace rr {

constexpr int kShadeBlock = 256;
constexpr float kBoxInflate = 1.00000036f;  // 1 + 2 gamma_3 (robust slab test, Ize 2013)

// ---------------------------------------------------------------------------
// beam axis angle 2 pi a / n with an exact quadrant reduction; returns (cos, sin)
__device__ __forceinline__ float2 beam_angle(uint32_t a, uint32_t n) {
  const uint32_t m = 4u * a;
  const uint32_t q = (m + n / 2u) / n;              // nearest quarter turn
  const int rem = (int)m - (int)(q * n);            // in [-n/2, n/2]
  float s, c;
  sincospif(0.5f * (float)rem / (float)n, &s, &c);
  switch (q & 3u) {
    case 0: return make_float2(c, s);
    case 1: return make_float2(-s, c);
    case 2: return make_float2(-c, -s);
    default: return make_float2(s, -c);
  }
}

// world direction of beam az's axis for a scan
__device__ __forceinline__ float3 beam_axis(const ScanDesc* sd, uint32_t az) {
  const float2 cs = beam_angle(az, __ldg(&sd->dims.x));
  float se, ce;
  sincosf(__ldg(&sd->beam.z), &se, &ce);
  return qrot(__ldg(&sd->quat), make_float3(ce * cs.x, ce * cs.y, se));
}

// Eq. 2: sigma = (b / 2) / (sqrt(2) erfinv(P))
__device__ __forceinline__ float d3_sigma(float b, float P) {
  return b > 0.0f ? 0.5f * b / (1.41421356237309515f * erfinvf(P)) : 0.0f;
}

// ---------------------------------------------------------------------------
// raygen: ray (az, k) of the D3 cone of its scan, energy 1 / N_s
__global__ void k_raygen(ScanArgs a) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    ScanCounters* c = a.ctr;
    for (int b = 0; b <= (int)RR_MAX_BOUNCES; ++b) {
      c->count[b] = 0;
      c->rec_start[b] = 0;
      c->seg_start[b] = 0;
    }
    for (int b = 0; b < (int)RR_MAX_BOUNCES; ++b) {
      c->trace_ticket[b] = 0;
      c->shade_ticket[b] = 0;
      c->vis_count[b] = 0;
      c->vis_ticket[b] = 0;
    }
    c->count[0] = a.n_rays0;
    c->stat_scans += (unsigned long long)a.n_scans;
  }
  if (i >= a.n_rays0) return;
  const uint32_t scan = owner_of(a.ray0, a.n_scans, i);
  const ScanDesc* sd = a.desc + scan;
  const uint32_t ns = __ldg(&sd->dims.y);
  const uint32_t local = i - __ldg(&a.ray0[scan]);
  const uint32_t az_l = local / ns, k = local - az_l * ns;
  const uint32_t az = __ldg(&sd->offs.w) + az_l;   // a scan may trace a range of the azimuths
  const float4 beam = __ldg(&sd->beam);
  const uint4 x = draw(__ldg(&sd->rng), az, k, 0u);
  const float u0 = u01(x.x), u1 = u01(x.y), u2 = u01(x.z);
  const float gauss = sqrtf(-2.0f * logf(u0)) * cospif(2.0f * u1);
  const float r = d3_sigma(beam.x, beam.y) * gauss;
  float sw, cw;
  sincospif(2.0f * u2 - 1.0f, &sw, &cw);      // omega = pi (2 u2 - 1)
  const float daz = r * cw, dinc = r * sw * __ldg(&sd->ext.x);   // elliptic beams: inclination stretched
  const float2 ph = beam_angle(az, __ldg(&sd->dims.x));
  float sd_, cd;
  sincosf(daz, &sd_, &cd);
  const float ca = ph.x * cd - ph.y * sd_, sa = ph.y * cd + ph.x * sd_;   // cos, sin of phi + daz
  float si, ci;
  sincosf(beam.z + dinc, &si, &ci);
  const float3 d = normalize(qrot(__ldg(&sd->quat), make_float3(ci * ca, ci * sa, si)));
  const bool masked = a.mask != nullptr && a.mask[i] != 0;
  const float4 pr = __ldg(&sd->pos_rmax);
  RayRec ray;
  ray.o_L = make_float4(pr.x, pr.y, pr.z, 0.0f);
  ray.d_E = make_float4(d.x, d.y, d.z, 1.0f / (float)ns);
  ray.meta = make_uint4(kNone, (az << 16) | k, masked ? 0x80000000u : 0u, (scan << 16) | kAir);
  a.rays[0][i] = ray;
}

// ---------------------------------------------------------------------------
// traversal
struct WoopRay {
  float3 o;            // origin in the frame (kx, ky, kz)
  float Sx, Sy, Sz;    // shear: d_kx / d_kz, d_ky / d_kz, 1 / d_kz
  uint32_t rot;        // the rotated triangle copy whose coordinates are in that frame
};

// The frame's third axis kz is the dominant axis of d; kx and ky follow it
// cyclically (kx = kz + 1, ky = kz + 2 mod 3), which is the triangle copy
// rotated by (kz + 1) mod 3.  Woop et al. swap kx and ky when d_kz < 0 to keep
// the winding; the test below accepts both windings, and swapping the two
// axes negates U, V, W, det and T exactly (each is a difference of the same
// rounded products, or a sum of such terms), so t and the decision are the
// same bit for bit without the swap.
__device__ __forceinline__ WoopRay make_woop(float3 o, float3 d) {
  WoopRay w;
  const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  const uint32_t kz = (ax >= ay && ax >= az) ? 0u : (ay >= az ? 1u : 2u);
  w.rot = kz == 2u ? 0u : kz + 1u;
  const float3 dr = tri_rotate(d, w.rot);
  w.o = tri_rotate(o, w.rot);
  w.Sx = dr.x / dr.z;
  w.Sy = dr.y / dr.z;
  w.Sz = 1.0f / dr.z;
  return w;
}

// watertight test; returns t (or -1) -- products are kept unfused so that a
// shared edge evaluates to exactly opposite values in both triangles
// (the vertices in the ray's frame: the triangle copy w.rot)
__device__ __forceinline__ float woop_hit(const WoopRay& w, float3 v0, float3 v1, float3 v2) {
  const float3 A = v0 - w.o, B = v1 - w.o, C = v2 - w.o;
  const float Az_ = A.z, Bz_ = B.z, Cz_ = C.z;
  const float Ax = __fsub_rn(A.x, __fmul_rn(w.Sx, Az_));
  const float Ay = __fsub_rn(A.y, __fmul_rn(w.Sy, Az_));
  const float Bx = __fsub_rn(B.x, __fmul_rn(w.Sx, Bz_));
  const float By = __fsub_rn(B.y, __fmul_rn(w.Sy, Bz_));
  const float Cx = __fsub_rn(C.x, __fmul_rn(w.Sx, Cz_));
  const float Cy = __fsub_rn(C.y, __fmul_rn(w.Sy, Cz_));
  const float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  const float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  const float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return -1.0f;
  const float det = U + V + W;
  if (det == 0.0f) return -1.0f;
  const float T = U * (w.Sz * Az_) + V * (w.Sz * Bz_) + W * (w.Sz * Cz_);
  return T / det;
}

// ---------------------------------------------------------------------------
// Resumable traversal.  A query (closest hit, or any hit for visibility) is
// advanced one step at a time -- one node visit or one triangle test -- so
// that a lane whose query has ended can take the next one while the other
// lanes of its warp go on.
//
// Closest hit: t_min < t < t_best on entry, (t, original id)
// lexicographically smallest.  Any hit: the first t_min < t < t_best.  The
// leaf `skip` (the one the ray starts on) is never reported.
struct Trav {
  float3 c0, c1;        // slab offsets (trav_begin): binary nodes, of the lower / upper box planes;
                        // wide nodes, of the near / far planes
  WoopRay w;            // the watertight-test frame
  float3 id;            // 1 / direction, zero components replaced by +-1e-30
  float t_min, t_best;
  uint32_t skip;
  uint32_t node;        // binary: next node; both: kNone once the query has ended
  uint32_t best, best_id, visits;
  uint32_t oct;                               // wide: direction octant
  uint32_t g_base, g_bits;                    // wide: node group
  uint32_t t_base, t_bits;                    // wide: triangles still to test, bit i = triangle t_base + i
  int sp;
};

__device__ __forceinline__ void trav_begin(Trav& s, float3 o, float3 d, float t_min, float t_best, uint32_t skip,
                                           uint32_t n_tris, bool wide) {
  s.w = make_woop(o, d);
  s.id = make_float3(1.0f / (fabsf(d.x) > 1e-30f ? d.x : copysignf(1e-30f, d.x)),
                     1.0f / (fabsf(d.y) > 1e-30f ? d.y : copysignf(1e-30f, d.y)),
                     1.0f / (fabsf(d.z) > 1e-30f ? d.z : copysignf(1e-30f, d.z)));
  // Slab test with one fma per plane: plane b is reached at t = fma(b, id, c)
  // with c = -(o id) -+ eps, where the robust form (b - o) id needs two
  // operations.  The fma form errs against (b - o) id by at most u |o id|
  // (o id rounded) + u |c| (c rounded) + u |t| (the fma itself), u = 2^-24.
  // eps = 4 u |o id| moves every near plane down and every far plane up by
  // more than the first two; the last is relative, like the errors of the
  // robust form, and the far-plane inflation kBoxInflate covers it.  So a box
  // the robust test accepts is accepted here too.
  {
    const float ox = __fmul_rn(o.x, s.id.x), oy = __fmul_rn(o.y, s.id.y), oz = __fmul_rn(o.z, s.id.z);
    float ex = 0x1p-22f * fabsf(ox), ey = 0x1p-22f * fabsf(oy), ez = 0x1p-22f * fabsf(oz);
    if (!wide) {   // the lower plane is the near one for a positive direction component
      ex = copysignf(ex, s.id.x);
      ey = copysignf(ey, s.id.y);
      ez = copysignf(ez, s.id.z);
    }
    s.c0 = make_float3(-ox - ex, -oy - ey, -oz - ez);
    s.c1 = make_float3(-ox + ex, -oy + ey, -oz + ez);
  }
  s.t_min = t_min;
  s.t_best = t_best;
  s.skip = skip;
  s.best = kNone;
  s.best_id = 0u;
  s.visits = 0u;
  s.sp = 0;
  if (wide) {
    s.oct = (s.id.x < 0.0f ? 1u : 0u) | (s.id.y < 0.0f ? 2u : 0u) | (s.id.z < 0.0f ? 4u : 0u);
    s.g_base = 0u;
    s.g_bits = (1u << 8) | (1u << s.oct);   // the root: internal slot 0 of a virtual group
    s.t_base = 0u;
    s.t_bits = 0u;
    s.node = n_tris ? 0u : kNone;
  } else {
    s.node = n_tris == 0 ? kNone : (n_tris == 1 ? kLeafBit : 0u);
  }
}

// triangle j against the query; returns true when an any-hit query is answered
template <bool kAny>
__device__ __forceinline__ bool trav_tri(Trav& s, const ScanArgs& a, uint32_t j, uint32_t& n_tris, bool count) {
  if (j == s.skip) return false;
  if (count) ++n_tris;
  const float4* tp = a.tri + a.tri_copy * s.w.rot + 3 * (size_t)j;
  const float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
  const float t = woop_hit(s.w, f3(v0), f3(v1), f3(v2));
  if (t > s.t_min) {
    if (kAny) {
      if (t < s.t_best) {
        s.best = j;
        return true;
      }
    } else {
      const uint32_t tid = __float_as_uint(v0.w);
      if (t < s.t_best || (t == s.t_best && s.best != kNone && tid < s.best_id)) {
        s.t_best = t;
        s.best = j;
        s.best_id = tid;
      }
    }
  }
  return false;
}

// one step over the binary LBVH (both children tested, nearer first)
template <bool kAny>
__device__ __forceinline__ void step_binary(Trav& s, uint32_t* stack, const ScanArgs& a, uint32_t& n_nodes,
                                            uint32_t& n_tris, bool count) {
  const uint32_t node = s.node;
  if (!(node & kLeafBit)) {
    if (count) ++n_nodes;
    ++s.visits;   // bounded where the query loop looks at its lanes
    const float3 id = s.id, cl = s.c0, ch = s.c1;
    const float4* np = a.nodes + 4 * (size_t)node;
    const float4 n0 = __ldg(np), n1 = __ldg(np + 1), n2 = __ldg(np + 2), n3 = __ldg(np + 3);
    // child 0
    float t0 = fmaf(n0.x, id.x, cl.x), t1 = fmaf(n0.y, id.x, ch.x);
    float lo0 = fminf(t0, t1), hi0 = fmaxf(t0, t1);
    t0 = fmaf(n0.z, id.y, cl.y);
    t1 = fmaf(n0.w, id.y, ch.y);
    lo0 = fmaxf(lo0, fminf(t0, t1));
    hi0 = fminf(hi0, fmaxf(t0, t1));
    t0 = fmaf(n2.x, id.z, cl.z);
    t1 = fmaf(n2.y, id.z, ch.z);
    lo0 = fmaxf(fmaxf(lo0, fminf(t0, t1)), s.t_min);
    hi0 = fminf(fminf(hi0, fmaxf(t0, t1)) * kBoxInflate, s.t_best);
    // child 1
    t0 = fmaf(n1.x, id.x, cl.x);
    t1 = fmaf(n1.y, id.x, ch.x);
    float lo1 = fminf(t0, t1), hi1 = fmaxf(t0, t1);
    t0 = fmaf(n1.z, id.y, cl.y);
    t1 = fmaf(n1.w, id.y, ch.y);
    lo1 = fmaxf(lo1, fminf(t0, t1));
    hi1 = fminf(hi1, fmaxf(t0, t1));
    t0 = fmaf(n2.z, id.z, cl.z);
    t1 = fmaf(n2.w, id.z, ch.z);
    lo1 = fmaxf(fmaxf(lo1, fminf(t0, t1)), s.t_min);
    hi1 = fminf(fminf(hi1, fmaxf(t0, t1)) * kBoxInflate, s.t_best);
    const bool h0 = lo0 <= hi0, h1 = lo1 <= hi1;
    const uint32_t c0 = __float_as_uint(n3.x), c1 = __float_as_uint(n3.y);
    // the nearer hit child next, the farther one pushed when both are hit,
    // else the next stack entry: selects and a predicated store instead of
    // branches, so that the lanes of a warp take the same path here
    const bool both = h0 && h1;
    const bool first0 = !h1 || (h0 && lo0 <= lo1);
    const uint32_t near = first0 ? c0 : c1, far = first0 ? c1 : c0;
    const int sp = s.sp;
    if (both && sp < kStack) stack[sp] = far;   // a predicated store: every local store costs an L2 sector
    if (both && sp >= kStack) atomicOr(&a.ctr->error, kErrStack);
    const int sp1 = sp + ((both && sp < kStack) ? 1 : 0);
    if (h0 || h1) {
      s.sp = sp1;
      s.node = near;
    } else {
      s.node = sp1 ? stack[sp1 - 1] : kNone;
      s.sp = sp1 ? sp1 - 1 : 0;
    }
    return;
  } else if (trav_tri<kAny>(s, a, node & ~kLeafBit, n_tris, count)) {
    s.node = kNone;
    return;
  }
  s.node = s.sp ? stack[--s.sp] : kNone;
}

// One step over the 8-wide quantised BVH: a triangle of the current
// triangle group, else the next child of the current node group, else a
// group from the stack.  A leaf slot holds 1..3 consecutive triangles (its
// count in two bits of the node's word w1.w); the hit leaf slots of a node
// become one mask over its up to 24 triangles.  Children are visited in slot order k ^ octant
// (near first) through node groups as in Ylitie, Karras, Laine, "Efficient
// incoherent ray traversal on GPUs through compressed wide BVHs" (HPG 2017):
// a group is (first child, internal-slot mask << 8 | hit children still to
// visit, bit k for slot k ^ octant), so one stack entry stands for up to 7
// pending children.  Slot boxes are decoded exactly (see kWideNodeWords);
// each contains the box of the binary node it stands for, and both node
// formats take the conservative slab test of trav_begin, so a query reaches
// every triangle it can hit in either BVH and finds the same closest hit.
template <bool kAny>
__device__ __forceinline__ void step_wide(Trav& s, uint2* stack, const ScanArgs& a, uint32_t& n_nodes,
                                          uint32_t& n_tris, bool count) {
  const uint32_t oct = s.oct;
  if (s.t_bits) {
    const uint32_t j = s.t_base + (uint32_t)__ffs(s.t_bits) - 1u;
    s.t_bits &= s.t_bits - 1u;
    if (j < a.n_tris && trav_tri<kAny>(s, a, j, n_tris, count)) s.node = kNone;
    return;
  }
  if (s.g_bits & 0xFFu) {
    const uint32_t k = __ffs(s.g_bits & 0xFFu) - 1u;
    s.g_bits &= ~(1u << k);
    const uint32_t slot = k ^ oct;
    const uint32_t node = s.g_base + __popc((s.g_bits >> 8) & ((1u << slot) - 1u));
    if (s.g_bits & 0xFFu) {
      if (s.sp < kStack) stack[s.sp++] = make_uint2(s.g_base, s.g_bits);
      else atomicOr(&a.ctr->error, kErrStack);
    }
    if (node >= a.node_cap) {   // only a failed build can get here
      atomicOr(&a.ctr->error, kErrBvh);
      s.node = kNone;
      return;
    }
    if (count) ++n_nodes;
    ++s.visits;   // bounded where the query loop looks at its lanes
    const float3 id = s.id, cn = s.c0, cf = s.c1;
    const bool neg_x = id.x < 0.0f, neg_y = id.y < 0.0f, neg_z = id.z < 0.0f;
    const uint4* np = reinterpret_cast<const uint4*>(a.nodes) + kWideNodeWords * (size_t)node;
    const uint4 w0 = __ldg(np), w1 = __ldg(np + 1), w2 = __ldg(np + 2), w3 = __ldg(np + 3), w4 = __ldg(np + 4);
    const float px = __uint_as_float(w0.x), py = __uint_as_float(w0.y), pz = __uint_as_float(w0.z);
    const float sx = __uint_as_float((w0.w & 0xFFu) << 23), sy = __uint_as_float(((w0.w >> 8) & 0xFFu) << 23),
                sz = __uint_as_float(((w0.w >> 16) & 0xFFu) << 23);
    const uint32_t imask = w0.w >> 24, valid = w1.z, counts = w1.w;
    // near and far plane bytes per axis: (lo, hi) for a positive direction, swapped otherwise
    const uint32_t nx0 = neg_x ? w3.z : w2.x, nx1 = neg_x ? w3.w : w2.y;
    const uint32_t fx0 = neg_x ? w2.x : w3.z, fx1 = neg_x ? w2.y : w3.w;
    const uint32_t ny0 = neg_y ? w4.x : w2.z, ny1 = neg_y ? w4.y : w2.w;
    const uint32_t fy0 = neg_y ? w2.z : w4.x, fy1 = neg_y ? w2.w : w4.y;
    const uint32_t nz0 = neg_z ? w4.z : w3.x, nz1 = neg_z ? w4.w : w3.y;
    const uint32_t fz0 = neg_z ? w3.x : w4.z, fz1 = neg_z ? w3.y : w4.w;
    uint32_t hit_i = 0u, tmask = 0u, first = 0u;   // first: the slot's first triangle (of the node's)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      // bits 0x4B0000qq = 2^23 + q (byte q of the word), decoded to P + q s exactly
      const uint32_t sel = 0x7440u | (uint32_t)(j & 3);
      const float bnx = fmaf(__uint_as_float(__byte_perm(j < 4 ? nx0 : nx1, 0x4B000000u, sel)), sx, px);
      const float bfx = fmaf(__uint_as_float(__byte_perm(j < 4 ? fx0 : fx1, 0x4B000000u, sel)), sx, px);
      const float bny = fmaf(__uint_as_float(__byte_perm(j < 4 ? ny0 : ny1, 0x4B000000u, sel)), sy, py);
      const float bfy = fmaf(__uint_as_float(__byte_perm(j < 4 ? fy0 : fy1, 0x4B000000u, sel)), sy, py);
      const float bnz = fmaf(__uint_as_float(__byte_perm(j < 4 ? nz0 : nz1, 0x4B000000u, sel)), sz, pz);
      const float bfz = fmaf(__uint_as_float(__byte_perm(j < 4 ? fz0 : fz1, 0x4B000000u, sel)), sz, pz);
      const float lo =
          fmaxf(fmaxf(fmaf(bnx, id.x, cn.x), fmaf(bny, id.y, cn.y)), fmaxf(fmaf(bnz, id.z, cn.z), s.t_min));
      const float hi = fminf(
          fminf(fminf(fmaf(bfx, id.x, cf.x), fmaf(bfy, id.y, cf.y)), fmaf(bfz, id.z, cf.z)) * kBoxInflate, s.t_best);
      const uint32_t c = counts >> (2 * j) & 3u;   // triangles of a leaf slot (0: inner or empty)
      if (lo <= hi && (valid >> j & 1u)) {
        if (imask >> j & 1u) hit_i |= 1u << (j ^ oct);
        else tmask |= ((1u << c) - 1u) << first;
      }
      first += c;
    }
    s.g_base = w1.x;
    s.g_bits = (imask << 8) | hit_i;
    s.t_base = w1.y;
    s.t_bits = tmask;
    return;
  }
  if (s.sp) {
    const uint2 e = stack[--s.sp];
    s.g_base = e.x;
    s.g_bits = e.y;
  } else {
    s.node = kNone;
  }
}

// ---------------------------------------------------------------------------
// Queries of one bounce.  kAny = false: the closest hit of every queued ray.
// kAny = true: the visibility test of the air-path return (Sec. III-A) for the
// candidates the shading pass listed (deferred visibility, which then settles
// the visible ones), or, with a min_energy cut, for the jobs k_vis_prep listed
// ahead of the shading pass.  Persistent: a warp claims jobs in chunks and hands
// them to its idle lanes once at least `refill` lanes are idle (or all are),
// so the lanes stay busy however uneven the query lengths are.
constexpr uint32_t kClaim = 32;

// Receive-beam weight of a return from p (Sec. III-A air path): g =
// exp(-delta^2 / 2 sigma^2), delta the angle between p - sensor and the beam
// axis of azimuth az; an elliptic beam scales the spread along the offset's
// direction around the axis.
__device__ __forceinline__ float rx_weight(const ScanDesc* sd, uint32_t az, float3 p) {
  const float4 beam = __ldg(&sd->beam);
  const float sigma = d3_sigma(beam.x, beam.y);
  const float3 v = p - f3(__ldg(&sd->pos_rmax));
  const float delta = angle_between(v, beam_axis(sd, az));
  float q = (delta / sigma) * (delta / sigma);
  const float aspect = __ldg(&sd->ext.x);
  if (aspect != 1.0f) {
    const float2 cs = beam_angle(az, __ldg(&sd->dims.x));
    float se, ce;
    sincosf(beam.z, &se, &ce);
    const float4 qt = __ldg(&sd->quat);
    const float3 ea = qrot(qt, make_float3(-cs.y, cs.x, 0.0f));
    const float3 ee = qrot(qt, make_float3(-se * cs.x, -se * cs.y, ce));
    const float c_a = dot(v, ea), c_e = dot(v, ee);
    const float perp2 = c_a * c_a + c_e * c_e;
    if (perp2 > 0.0f) q *= (c_a * c_a + c_e * c_e / (aspect * aspect)) / perp2;
  }
  return sigma > 0.0f ? expf(-0.5f * q) : 0.0f;
}

// Deferred visibility: the sensor is visible from candidate i of a bounce,
// so its air-path return is taken (Sec. III-A; returns deplete the ray): the
// reserved record gets its energy and the child it depletes (or, when the
// child was not spawned, the terminated tally) loses it; the debug dump and
// tallies are patched like the shading pass would have written them.
__device__ __noinline__ void settle_air_path(const ScanArgs& a, uint32_t bounce, uint32_t i) {
  const VisJob* jp = reinterpret_cast<const VisJob*>(a.rays[bounce & 1]) + i;
  const uint4 ix = jp->idx;
  const float4 v = jp->val;
  const float e_child = fmaxf(v.x - v.y, 0.0f);
  if (ix.y != kNone) a.rays[(bounce + 1) & 1][ix.y].d_E.w = e_child;
  if (ix.z != kNone) a.recs[ix.z].y = __float_as_uint(v.z);
  if (ix.w != kNone && a.tallies != nullptr) {
    float* tp = a.tallies + 4 * (size_t)ix.w;
    atomicAdd(tp, v.y);
    if (ix.y == kNone) atomicAdd(tp + 3, e_child - fmaxf(v.x, 0.0f));
  }
  const uint32_t si = __float_as_uint(v.w);
  if (si != kNone && a.segs != nullptr && si < a.seg_cap) {
    a.segs[si].flags |= 2u;
    a.segs[si].ret_a = v.y;
  }
}

// Steps a busy lane takes between two looks at the warp's idle lanes.  The
// look (votes, the refill hand-out, the end-of-query test) costs about a
// fifth of a node visit's instructions when taken every step; taking it every
// kSteps steps lets a lane whose query ended idle for at most kSteps steps
// (campus bench step: 1.85 ms at 1, 1.77 at 4, 1.73 from 12 to 64).
constexpr int kSteps = 16;
// kCount: the traversal counters (RR_COUNT_TRAVERSAL) are compiled only into
// the kernels of the scans that ask for them
template <bool kAny, int kBlock, bool kWide, bool kCount>
__global__ void __launch_bounds__(kBlock) k_query(ScanArgs a, uint32_t bounce) {
  typedef typename std::conditional<kWide, uint2, uint32_t>::type StackEntry;
  ScanCounters* C = a.ctr;
  const uint32_t n = kAny ? C->vis_count[bounce] : C->count[bounce];
  uint32_t* ticket = kAny ? &C->vis_ticket[bounce] : &C->trace_ticket[bounce];
  const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  if (!kAny) {
    const uint32_t tiles = (n + kShadeBlock - 1) / kShadeBlock;
    for (uint32_t t = gtid; t < tiles; t += gsz) a.tile_status[t] = 0ull;
    // the shading pass of this bounce counts the next bounce's rays per order bucket
    if (a.order_hist != nullptr && bounce + 1 <= RR_MAX_BOUNCES)
      for (uint32_t t = gtid; t < kOrderBuckets; t += gsz) a.order_hist[(bounce + 1) * kOrderBuckets + t] = 0u;
  }
  const uint32_t* __restrict__ perm = (!kAny && bounce > 0) ? a.order_perm : nullptr;
  const RayRec* __restrict__ q = a.rays[bounce & 1];
  const uint2* __restrict__ jobs = reinterpret_cast<const uint2*>(a.rays[(bounce + 1) & 1]);
  // after a failed build every query ends at once as a miss and the scan fails
  const bool bvh_ok = (a.bvh_status == nullptr || *a.bvh_status == 0u) &&
                      (a.build_status == nullptr || (*a.build_status & kErrTopBuild) == 0u);
  if (!bvh_ok && gtid == 0) atomicOr(&C->error, kErrBvh);
  constexpr bool count = kCount;
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t refill = a.refill;
  Trav s;
  s.node = kNone;
  StackEntry stack[kStack];
  uint32_t ray_i = kNone;   // ray of the lane's query (kNone: idle)
  float wa = 0.0f;          // any hit: W(omega_a) of the candidate
  uint32_t c_base = 0u, c_end = 0u;   // claimed, unassigned jobs (warp-uniform)
  bool exhausted = false;             // the job list is used up (warp-uniform)
  uint32_t n_done = 0, n_nodes = 0, n_tris = 0;
  while (true) {
    const bool idle = ray_i == kNone;
    const uint32_t im = __ballot_sync(0xFFFFFFFFu, idle);
    if (im != 0u && !exhausted && ((uint32_t)__popc(im) >= refill || im == 0xFFFFFFFFu)) {
      const uint32_t need = (uint32_t)__popc(im), rank = (uint32_t)__popc(im & lt);
      const uint32_t avail = c_end - c_base;
      uint32_t job = kNone;
      if (idle && rank < avail) job = c_base + rank;
      if (need <= avail) {
        c_base += need;
      } else {
        c_base = c_end;
        const uint32_t more = need - avail, chunk = max(more, kClaim);
        uint32_t b = 0;
        if (lane == 0) b = atomicAdd(ticket, chunk);
        b = __shfl_sync(0xFFFFFFFFu, b, 0);
        if (b >= n) {
          exhausted = true;
        } else {
          const uint32_t e = (n - b > chunk) ? b + chunk : n;
          if (idle && rank >= avail && b + (rank - avail) < e) job = b + (rank - avail);
          c_base = min(b + more, e);
          c_end = e;
        }
      }
      if (job != kNone) {
        if (kAny && a.defer_vis) {
          ray_i = a.vis_list[job];
          const float4 pl = reinterpret_cast<const VisJob*>(q)[ray_i].p_leaf;
          const uint32_t scan = min(reinterpret_cast<const VisJob*>(q)[ray_i].idx.x, a.n_scans - 1u);
          const ScanDesc* sd = a.desc + scan;
          const float3 p = f3(pl);
          const float3 v = f3(__ldg(&sd->pos_rmax)) - p;
          const float dist = length(v);
          trav_begin(s, p, (1.0f / dist) * v, __ldg(&sd->phys.x), dist, __float_as_uint(pl.w), a.n_tris, kWide);
        } else if (kAny) {
          const uint2 jb = jobs[job];
          ray_i = jb.x;
          wa = __uint_as_float(jb.y);
          const RayRec ray = q[ray_i];
          const HitRec h = a.hits[ray_i];
          const uint2 sm = ray_scan_medium(a, ray.meta.w);
          const ScanDesc* sd = a.desc + sm.x;
          const float3 o = f3(ray.o_L), d = f3(ray.d_E);
          const float3 p = o + h.t * d;
          const float3 v = f3(__ldg(&sd->pos_rmax)) - p;
          const float dist = length(v);
          trav_begin(s, p, (1.0f / dist) * v, __ldg(&sd->phys.x), dist, h.leaf, a.n_tris, kWide);
        } else {
          ray_i = perm ? perm[job] : job;
          if (ray_i >= n) ray_i = job;   // only after a failed shading pass (the scan reports it)
          const RayRec ray = q[ray_i];
          const uint2 sm = ray_scan_medium(a, ray.meta.w);
          const float4 phys = __ldg(&a.desc[sm.x].phys);   // t_min, min_energy, freq, r_lim
          const float n_cur = sm.y == kAir ? 1.0f : __ldg(&a.mats[sm.y].n);
          // past t_lim no return can reach the image
          trav_begin(s, f3(ray.o_L), f3(ray.d_E), phys.x, (phys.w - ray.o_L.w) / n_cur, ray.meta.x, a.n_tris,
                     kWide);
        }
        if (!bvh_ok) s.node = kNone;
      }
    }
    const bool busy = ray_i != kNone;
    if (!__any_sync(0xFFFFFFFFu, busy)) {
      if (exhausted) break;
      continue;
    }
    if (busy) {
#pragma unroll 2
      for (int u = 0; u < kSteps && s.node != kNone; ++u) {
        if (kWide) step_wide<kAny>(s, reinterpret_cast<uint2*>(stack), a, n_nodes, n_tris, count);
        else step_binary<kAny>(s, reinterpret_cast<uint32_t*>(stack), a, n_nodes, n_tris, count);
      }
      // depth-first traversal of a tree visits each of its internal nodes
      // (fewer than n_tris, binary or wide) at most once: more visits mean a
      // malformed hierarchy (checked here, at most kSteps visits late)
      if (s.node != kNone && s.visits > a.n_tris) {
        atomicOr(&a.ctr->error, kErrBvh);
        s.node = kNone;
      }
      if (s.node == kNone) {   // the query has ended
        if (kAny && a.defer_vis) {
          if (s.best == kNone) settle_air_path(a, bounce, ray_i);
        } else if (kAny) {
          HitRec* hp = a.hits + ray_i;
          uint32_t fl = hp->flags | 1u;
          float wag = 0.0f;
          if (s.best == kNone) {   // the sensor is visible from the hit point: its window W
            fl |= 2u;               // (the receive weight g is applied where the return is made)
            wag = wa;
          }
          hp->flags = fl;
          hp->wa_g = wag;
        } else {
          HitRec h;
          h.t = s.best == kNone ? INFINITY : s.t_best;
          h.leaf = s.best;
          h.flags = min(s.visits, 0xFFFFFFu) << 8;   // bits 8..31: node visits (diagnostics)
          h.wa_g = 0.0f;
          a.hits[ray_i] = h;
        }
        ++n_done;
        ray_i = kNone;
      }
    }
  }
  // counters, one atomic per warp
  for (int off = 16; off > 0; off >>= 1) n_done += __shfl_xor_sync(0xFFFFFFFFu, n_done, off);
  if (lane == 0 && n_done) atomicAdd(kAny ? &C->stat_anyhit : &C->stat_closest, (unsigned long long)n_done);
  if (count) {
    unsigned long long nn = n_nodes, nt = n_tris;
    for (int off = 16; off > 0; off >>= 1) {
      nn += __shfl_xor_sync(0xFFFFFFFFu, nn, off);
      nt += __shfl_xor_sync(0xFFFFFFFFu, nt, off);
    }
    if (lane == 0) {
      atomicAdd(kAny ? &C->stat_nodes_any : &C->stat_nodes, nn);
      atomicAdd(kAny ? &C->stat_tris_any : &C->stat_tris, nt);
    }
  }
}

// Candidates of the air-path return (Sec. III-A) at bounce >= 1: the mean
// reflection direction (or, leaving a medium into air, the refracted one)
// against the direction to the sensor, through the beam window of the lobe.
// Rays whose window is open become jobs (ray, W) of the visibility query,
// appended with one atomic per warp into the free ray buffer of the next
// bounce (order does not matter: each job names its ray).
__global__ void __launch_bounds__(256) k_vis_prep(ScanArgs a, uint32_t bounce) {
  ScanCounters* C = a.ctr;
  const uint32_t n = C->count[bounce];
  const RayRec* __restrict__ q = a.rays[bounce & 1];
  uint2* __restrict__ jobs = reinterpret_cast<uint2*>(a.rays[(bounce + 1) & 1]);
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t warp0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u, wstride = gridDim.x * blockDim.x;
  for (uint32_t base = warp0; base < n; base += wstride) {
    const uint32_t i = base + lane;
    bool want = false;
    float wa = 0.0f;
    if (i < n) {
      const HitRec h = a.hits[i];
      if (h.leaf != kNone && h.leaf < a.n_tris) {
        const RayRec ray = q[i];
        const uint2 sm = ray_scan_medium(a, ray.meta.w);
        const uint32_t medium = sm.y;
        const ScanDesc* sd = a.desc + sm.x;
        if (__ldg(&sd->rng.w) & RR_MULTIPATH) {
          const float3 o = f3(ray.o_L), d = f3(ray.d_E);
          const float n_cur = medium == kAir ? 1.0f : __ldg(&a.mats[medium].n);
          const float4 nr = __ldg(a.tri + (size_t)kTriCopies * a.tri_copy + h.leaf);   // unit normal, material
          const uint32_t mid = __float_as_uint(nr.w);
          const MatDev m = a.mats[mid];
          float3 nrm = f3(nr);
          float cos_i = -dot(d, nrm);
          const bool entering = cos_i > 0.0f;
          float n2 = m.n;
          if (!entering) {
            nrm = -nrm;
            cos_i = -cos_i;
            n2 = 1.0f;
          }
          const float3 p = o + h.t * d;
          const float3 v = f3(__ldg(&sd->pos_rmax)) - p;
          const float side = dot(v, nrm);
          float3 dir_out = make_float3(0.f, 0.f, 0.f);
          bool cand = false;
          if (entering && medium == kAir) {
            dir_out = normalize(d + (2.0f * cos_i) * nrm);
            cand = side > 0.0f;
          } else if (!entering && medium != kAir && !m.pec) {
            const float eta = n_cur / n2;
            const float sin2_t = eta * eta * (1.0f - cos_i * cos_i);
            if (sin2_t < 1.0f) {
              const float cos_t = sqrtf(1.0f - sin2_t);
              dir_out = normalize(eta * d + (eta * cos_i - cos_t) * nrm);
              cand = side < 0.0f;
            }
          }
          if (cand) {   // as the deferred candidates: W and the receive weight g both non-zero
            wa = brdf_window(m, a.lut + (size_t)mid * (kLutCells + 1), angle_between(dir_out, v),
                             __ldg(&sd->beam.x));
            want = wa > 0.0f && wa * rx_weight(sd, ray.meta.y >> 16, p) > 0.0f;
          }
        }
      }
    }
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, want);
    if (m) {
      uint32_t b = 0;
      if (lane == __ffs(m) - 1) b = atomicAdd(&C->vis_count[bounce], (uint32_t)__popc(m));
      b = __shfl_sync(0xFFFFFFFFu, b, __ffs(m) - 1);
      if (want) jobs[b + __popc(m & lt)] = make_uint2(i, __float_as_uint(wa));
    }
  }
}

// ---------------------------------------------------------------------------
// decoupled look-back over tiles: status word = flag << 62 | recs << 31 | kids
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagPre = 2ull << 62;
constexpr unsigned long long kMask31 = 0x7FFFFFFFull;

__device__ __forceinline__ unsigned long long ld_status(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_status(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// exclusive (kids, recs) prefix of tile `tile`, computed by one full warp
__device__ __forceinline__ uint2 look_back(const ScanArgs& a, uint32_t tile, uint32_t agg_kids, uint32_t agg_recs) {
  const int lane = threadIdx.x & 31;
  unsigned long long* st = a.tile_status;
  const unsigned long long mine = ((unsigned long long)agg_recs << 31) | agg_kids;
  if (tile == 0) {
    if (lane == 0) st_status(st, kFlagPre | mine);
    return make_uint2(0u, 0u);
  }
  if (lane == 0) st_status(st + tile, kFlagAgg | mine);
  uint32_t ex_k = 0, ex_r = 0;
  int j = (int)tile - 1;
  uint32_t spins = 0;
  while (true) {
    const int idx = j - lane;
    unsigned long long s = idx >= 0 ? ld_status(st + idx) : kFlagPre;
    while (__any_sync(0xFFFFFFFFu, (s >> 62) == 0ull)) {
      if (++spins > kSpinLimit) {
        if (lane == 0) atomicOr(&a.ctr->error, kErrTimeout);
        s = kFlagPre;   // give up: the scan is reported as failed
        break;
      }
      if ((s >> 62) == 0ull) s = ld_status(st + idx);
    }
    const uint32_t pre = __ballot_sync(0xFFFFFFFFu, (s >> 62) == 2ull);
    const int first = pre ? __ffs(pre) - 1 : 32;
    const uint32_t vk = lane <= first ? (uint32_t)(s & kMask31) : 0u;
    const uint32_t vr = lane <= first ? (uint32_t)((s >> 31) & kMask31) : 0u;
    ex_k += __reduce_add_sync(0xFFFFFFFFu, vk);
    ex_r += __reduce_add_sync(0xFFFFFFFFu, vr);
    if (pre) break;
    j -= 32;
  }
  if (lane == 0)
    st_status(st + tile, kFlagPre | ((unsigned long long)(agg_recs + ex_r) << 31) | (agg_kids + ex_k));
  return make_uint2(ex_k, ex_r);
}

// failure detection: one warp runs the look-back of tile 1 while tile 0
// never publishes (its status word stays 0), so the bounded wait gives up
__global__ void k_selftest_look_back(ScanArgs a) { look_back(a, 1u, 0u, 0u); }

// ---------------------------------------------------------------------------
// query order: bucket of a queued ray (direction octant, then a 4 x 64 grid of
// cells of its origin around the sensor: height in r_max / 16 steps from one
// below the sensor, horizontal r_max / 4 cells in Morton order)
__device__ __forceinline__ uint32_t order_key(const ScanArgs& a, const RayRec& r) {
  const ScanDesc* sd = a.desc + ray_scan_medium(a, r.meta.w).x;
  const float4 pr = __ldg(&sd->pos_rmax);
  const float inv = 4.0f / fmaxf(pr.w, 1e-3f);
  const int cx = min(max((int)floorf((r.o_L.x - pr.x) * inv) + 4, 0), 7);
  const int cy = min(max((int)floorf((r.o_L.y - pr.y) * inv) + 4, 0), 7);
  const int cz = min(max((int)floorf((r.o_L.z - pr.z) * (4.0f * inv)) + 1, 0), 3);
  uint32_t xy = 0;
#pragma unroll
  for (int b = 0; b < 3; ++b) xy |= (((uint32_t)cx >> b) & 1u) << (2 * b) | (((uint32_t)cy >> b) & 1u) << (2 * b + 1);
  const uint32_t oct = (r.d_E.x < 0.0f ? 1u : 0u) | (r.d_E.y < 0.0f ? 2u : 0u) | (r.d_E.z < 0.0f ? 4u : 0u);
  return oct << 8 | (uint32_t)cz << 6 | xy;
}

// exclusive prefix of the bucket counts of a bounce (one block of 1024 threads, two buckets each)
__global__ void __launch_bounds__(1024) k_order_scan(ScanArgs a, uint32_t bounce) {
  __shared__ uint32_t s_w[32];
  const uint32_t* h = a.order_hist + bounce * kOrderBuckets;
  const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
  const uint32_t c0 = h[2 * t], c1 = h[2 * t + 1];
  uint32_t x = c0 + c1;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
    if ((int)lane >= off) x += y;
  }
  if (lane == 31u) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = s_w[lane];
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, v, off);
      if ((int)lane >= off) v += y;
    }
    s_w[lane] = v;
  }
  __syncthreads();
  const uint32_t excl = x - (c0 + c1) + (warp ? s_w[warp - 1] : 0u);
  a.order_off[2 * t] = excl;
  a.order_off[2 * t + 1] = excl + c0;
}

// the permutation: every queued ray of the bounce to a position of its
// bucket.  A block takes a contiguous chunk of the queue, counts its keys in
// shared memory, reserves each bucket's share with one atomic and places its
// rays (in any order within a bucket: every query's result is independent
// of the order)
__global__ void __launch_bounds__(256) k_order_place(ScanArgs a, uint32_t bounce) {
  __shared__ uint32_t s_cnt[kOrderBuckets];
  __shared__ uint32_t s_base[kOrderBuckets];
  const uint32_t n = min(a.ctr->count[bounce], a.ray_cap);
  const uint32_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const uint32_t i0 = blockIdx.x * chunk, i1 = min(i0 + chunk, n);
  for (uint32_t j = threadIdx.x; j < kOrderBuckets; j += blockDim.x) s_cnt[j] = 0u;
  __syncthreads();
  for (uint32_t i = i0 + threadIdx.x; i < i1; i += blockDim.x)
    atomicAdd(&s_cnt[a.order_key[i] & (kOrderBuckets - 1u)], 1u);
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < kOrderBuckets; j += blockDim.x) {
    const uint32_t c = s_cnt[j];
    s_base[j] = c ? atomicAdd(&a.order_off[j], c) : 0u;
    s_cnt[j] = 0u;
  }
  __syncthreads();
  for (uint32_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const uint32_t key = a.order_key[i] & (kOrderBuckets - 1u);
    const uint32_t pos = s_base[key] + atomicAdd(&s_cnt[key], 1u);
    if (pos < a.ray_cap) a.order_perm[pos] = i;
  }
}

// ---------------------------------------------------------------------------
// shade

// optional range weight of a return at range r (metres): (1 / r)^k for
// r > 1 m, k = the scan's range_falloff (Eq. 1's power falloff; 0: off)
__device__ __forceinline__ float range_weight(const ScanDesc* sd, float r) {
  const float k = __ldg(&sd->ext.w);
  return (k != 0.0f && r > 1.0f) ? powf(r, -k) : 1.0f;
}

// The shading pass runs with 3 resident blocks per SM (80 registers) or 4
// (64 registers, a few spilled).  Launch sequences with many rays take 4: the
// more warps hide more of the random triangle and material loads (5M-triangle
// city, 133k initial rays per sequence: 1.9 % per step).  Small ones take 3:
// there the launch holds fewer tiles than the SMs have room for, each tile's
// chain of dependent loads sets the time and the spills lengthen it (200k-
// triangle campus, 27k initial rays per sequence: 1.4 %).
constexpr uint32_t kShadeManyRays = 1u << 16;   // initial rays of a launch sequence

template <int kMinBlocks>
__global__ void __launch_bounds__(kShadeBlock, kMinBlocks) k_shade(ScanArgs a, uint32_t bounce) {
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_wsum[kShadeBlock / 32];
  __shared__ uint2 s_excl;
  extern __shared__ uint32_t s_hist[];   // [kOrderBuckets] children per order bucket (query order on only)
  const uint32_t n = a.ctr->count[bounce];
  const uint32_t tiles = (n + kShadeBlock - 1) / kShadeBlock;
  const uint32_t rec0 = a.ctr->rec_start[bounce];
  const uint32_t seg0 = a.ctr->seg_start[bounce];
  const RayRec* qin = a.rays[bounce & 1];   // not restrict: deferred visibility writes its jobs over it
  RayRec* __restrict__ qout = a.rays[(bounce + 1) & 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (n == 0) {
    // empty queue: no tile will publish the offsets of the next bounce
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.ctr->count[bounce + 1] = 0u;
      a.ctr->rec_start[bounce + 1] = rec0;
      a.ctr->seg_start[bounce + 1] = seg0;
    }
    return;
  }
  const bool counting = a.order_key != nullptr && bounce + 1 < a.max_bounces;
  if (counting)
    for (uint32_t j = threadIdx.x; j < kOrderBuckets; j += kShadeBlock) s_hist[j] = 0u;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&a.ctr->shade_ticket[bounce], 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= tiles) break;
    const uint32_t i = tile * kShadeBlock + threadIdx.x;
    RayRec kid[2];
    uint2 rec[2];
    uint32_t nk = 0, nr = 0;
    bool cand = false;           // an air-path candidate left to the visibility query (deferred visibility)
    int vj_kid = -1, vj_rec = -1;   // its child in kid[], its record in rec[] (-1: none)
    if (i < n) {
      const RayRec ray = qin[i];
      const HitRec h = a.hits[i];
      const uint32_t az = ray.meta.y >> 16, k = ray.meta.y & 0xFFFFu;
      const uint32_t path = ray.meta.z & 0x7FFFFFFFu;
      const bool masked = (ray.meta.z >> 31) != 0u;
      const uint2 sm = ray_scan_medium(a, ray.meta.w);
      const uint32_t scan = sm.x, medium = sm.y;
      const ScanDesc* sd = a.desc + scan;
      const uint4 dims = __ldg(&sd->dims);   // n_az, ns, max_bounces, n_bins
      const uint4 offs = __ldg(&sd->offs);   // first ray, first column
      const float E = ray.d_E.w;
      float tal[4] = {0.f, 0.f, 0.f, 0.f};
      float dbg_cos = 0.f, dbg_ret_t = 0.f, dbg_ret_a = 0.f;
      uint32_t orig = kNone;
      if (h.leaf == kNone || h.leaf >= a.n_tris) {
        tal[2] = E;   // escaped (or beyond the range limit); an index past the triangles only after a failed step
      } else {
        const float3 o = f3(ray.o_L), d = f3(ray.d_E);
        const float4 pr = __ldg(&sd->pos_rmax);
        const float4 beam = __ldg(&sd->beam);   // b, P, elevation, bin_size
        const float4 phys = __ldg(&sd->phys);   // t_min, min_energy, freq, r_lim
        const uint4 rng = __ldg(&sd->rng);
        const float3 s_pos = f3(pr);
        const bool deeper = bounce + 1 < dims.z;
        const float t = h.t;
        const float3 p = o + t * d;
        const float n_cur = medium == kAir ? 1.0f : a.mats[medium].n;
        const float L1 = ray.o_L.w + n_cur * t;
        float E1 = E;
        if (medium != kAir) {
          const float alpha = kPi * n_cur * a.mats[medium].tan_d * phys.z / kC0;
          E1 = E * expf(-2.0f * alpha * t);
          tal[1] = E - E1;
        }
        const float4 nrw = __ldg(a.tri + (size_t)kTriCopies * a.tri_copy + h.leaf);   // unit normal, material
        orig = __float_as_uint(__ldg(&a.tri[3 * (size_t)h.leaf].w));
        const uint32_t mid = __float_as_uint(nrw.w);
        const MatDev m = a.mats[mid];
        const float4* lut = a.lut + (size_t)mid * (kLutCells + 1);
        float3 nrm = f3(nrw);
        float cos_i = -dot(d, nrm);
        const bool entering = cos_i > 0.0f;
        float n2 = m.n;
        uint32_t next_med = mid;
        if (!entering) {
          nrm = -nrm;
          cos_i = -cos_i;
          n2 = 1.0f;
          next_med = kAir;
        }
        float R = 1.0f, T = 0.0f, cos_t = 0.0f;
        bool can_refract = false;
        const float eta = n_cur / n2;
        if (!m.pec) {
          const float sin2_t = eta * eta * (1.0f - cos_i * cos_i);
          if (sin2_t < 1.0f) {
            cos_t = sqrtf(1.0f - sin2_t);
            const float rs = (n_cur * cos_i - n2 * cos_t) / (n_cur * cos_i + n2 * cos_t);
            const float rp = (n_cur * cos_t - n2 * cos_i) / (n_cur * cos_t + n2 * cos_i);
            R = 0.5f * (rs * rs + rp * rp);
            T = 1.0f - R;
            can_refract = true;
          }
        }
        const float3 d_refl = normalize(d + (2.0f * cos_i) * nrm);
        // traveled-path return: omega = theta0 + theta1 = 2 theta0, range L1
        const float theta0 = angle_between(d, -nrm);
        const float ret_t = E1 * R * fminf(brdf_window(m, lut, 2.0f * theta0, beam.x), 1.0f);
        float ret_a = 0.0f, range_a = 0.0f, e_rec = 0.0f;
        bool air_T = false;
        // the air-path candidate (Sec. III-A): its window W is open toward the
        // sensor; with deferred visibility it is found here, else the
        // visibility query has run and left W in the hit record when visible
        float wag = 0.0f;
        if (a.defer_vis) {
          if (bounce >= 1u && (rng.w & RR_MULTIPATH)) {
            const float3 v = s_pos - p;
            const float side = dot(v, nrm);
            float3 dir_out = d_refl;
            bool c = false;
            if (entering && medium == kAir) {
              c = side > 0.0f;
            } else if (!entering && medium != kAir && can_refract) {
              dir_out = normalize(eta * d + (eta * cos_i - cos_t) * nrm);
              c = side < 0.0f;
            }
            if (c) {   // a window closed toward the sensor, or a receive weight that is 0, returns nothing
              const float wa = brdf_window(m, lut, angle_between(dir_out, v), beam.x);
              if (wa > 0.0f) {
                wag = wa * rx_weight(sd, az, p);
                cand = wag > 0.0f;
              }
            }
          }
        } else if (h.wa_g > 0.0f) {
          wag = h.wa_g * rx_weight(sd, az, p);
        }
        if (wag > 0.0f) {
          float base, cap;
          if (entering && medium == kAir) {
            base = E1 * R;
            cap = E1 * R - ret_t;
          } else {
            air_T = true;
            base = E1 * T;
            cap = E1 * T;
          }
          ret_a = fmaxf(fminf(base * wag, cap), 0.0f);
          range_a = 0.5f * (L1 + length(s_pos - p));
        }
        // a candidate's return is taken once its visibility is known: until
        // then the ray gives nothing to the air path
        const float ret_a_now = cand ? 0.0f : ret_a;
        tal[0] = ret_t + ret_a_now;
        dbg_cos = cos_i;
        dbg_ret_t = ret_t;
        dbg_ret_a = ret_a_now;
        if (!masked) {
          if (ret_t > 0.0f) {
            const float bin = floorf(L1 / beam.w);
            if (bin < (float)dims.w) {
              float e = ret_t;
              if (rng.w & RR_SPECKLE) e *= -logf(u01(draw(rng, az, k, 1u | (((path << 8) | bounce) << 8)).x));
              e *= range_weight(sd, L1);
              rec[nr++] = make_uint2(((offs.y + az - offs.w) << kBinBits) | (uint32_t)bin, __float_as_uint(e));
            }
          }
          if (ret_a > 0.0f) {
            const float bin = floorf(range_a / beam.w);
            if (bin < (float)dims.w) {
              float e = ret_a;
              if (rng.w & RR_SPECKLE) e *= -logf(u01(draw(rng, az, k, 1u | (((path << 8) | bounce) << 8)).y));
              e *= range_weight(sd, range_a);
              if (cand) {   // reserved with energy 0, written if the sensor is visible
                e_rec = e;
                vj_rec = (int)nr;
              }
              rec[nr++] =
                  make_uint2(((offs.y + az - offs.w) << kBinBits) | (uint32_t)bin, cand ? 0u : __float_as_uint(e));
            }
          }
        }
        const float e_refl = fmaxf(E1 * R - ret_t - (air_T ? 0.0f : ret_a_now), 0.0f);
        const float e_refr = fmaxf(E1 * T - (air_T ? ret_a_now : 0.0f), 0.0f);
        const bool in_range = L1 < pr.w;
        const bool sp_refl = deeper && in_range && e_refl >= phys.y;
        const bool sp_refr = deeper && in_range && can_refract && (rng.w & RR_REFRACTION) && e_refr >= phys.y;
        if (!sp_refl) tal[3] += e_refl;
        if (!sp_refr) tal[3] += e_refr;
        const uint32_t mbit = ray.meta.z & 0x80000000u;
        if (sp_refl) {
          RayRec& c = kid[nk++];
          c.o_L = make_float4(p.x, p.y, p.z, L1);
          c.d_E = make_float4(d_refl.x, d_refl.y, d_refl.z, e_refl);
          c.meta = make_uint4(h.leaf, ray.meta.y, mbit | (path << 1), (scan << 16) | medium);
        }
        if (sp_refr) {
          const float3 d_refr = normalize(eta * d + (eta * cos_i - cos_t) * nrm);
          RayRec& c = kid[nk++];
          c.o_L = make_float4(p.x, p.y, p.z, L1);
          c.d_E = make_float4(d_refr.x, d_refr.y, d_refr.z, e_refr);
          c.meta = make_uint4(h.leaf, ray.meta.y, mbit | (path << 1) | 1u, (scan << 16) | next_med);
        }
        if (cand) {   // the job, over this ray's record (read above, not read again)
          vj_kid = air_T ? (sp_refr ? (sp_refl ? 1 : 0) : -1) : (sp_refl ? 0 : -1);
          VisJob j;
          j.p_leaf = make_float4(p.x, p.y, p.z, __uint_as_float(h.leaf));
          j.idx = make_uint4(scan, kNone, kNone,
                             a.tallies != nullptr ? offs.x + (az - offs.w) * dims.y + k : kNone);
          j.val = make_float4(air_T ? E1 * T : E1 * R - ret_t, ret_a, e_rec,
                              __uint_as_float(a.segs != nullptr ? seg0 + i : kNone));
          reinterpret_cast<VisJob*>(a.rays[bounce & 1])[i] = j;
        }
      }
      if (a.tallies != nullptr) {
        float* tp = a.tallies + 4 * ((size_t)offs.x + (size_t)(az - offs.w) * dims.y + k);
        for (int q = 0; q < 4; ++q)
          if (tal[q] != 0.0f) atomicAdd(tp + q, tal[q]);
      }
      if (a.segs != nullptr) {
        const uint32_t si = seg0 + i;
        if (si < a.seg_cap) {
          rr_segment sg;
          sg.az = az;
          sg.k = k;
          sg.path = path;
          sg.bounce = bounce;
          sg.tri = orig;
          sg.t = h.leaf == kNone ? INFINITY : h.t;
          sg.E = E;
          sg.flags = (h.flags & 0xFFu) | (cand ? 1u : 0u);   // bit 0: visibility tested, bit 1: visible
          sg.cos_i = dbg_cos;
          sg.ret_t = dbg_ret_t;
          sg.ret_a = dbg_ret_a;
          sg.visits = (float)(h.flags >> 8);   // node visits of the closest-hit query
          a.segs[si] = sg;
        } else {
          atomicOr(&a.ctr->error, kErrCapacitySegs);
        }
      }
    }
    // block scan of (kids, recs)
    const uint32_t packed = nk | (nr << 16);
    uint32_t x = packed;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    uint32_t wpre = 0, total = 0;
    for (int w2 = 0; w2 < kShadeBlock / 32; ++w2) {
      const uint32_t v = s_wsum[w2];
      if (w2 < warp) wpre += v;
      total += v;
    }
    const uint32_t local = x - packed + wpre;
    if (warp == 0) {
      const uint2 ex = look_back(a, tile, total & 0xFFFFu, total >> 16);
      if (lane == 0) s_excl = ex;
    }
    __syncthreads();
    const uint2 ex = s_excl;
    const uint32_t kbase = ex.x + (local & 0xFFFFu), rbase = ex.y + (local >> 16);
    if (a.defer_vis) {
      // the candidates' child and record positions, and the list of jobs
      // (one atomic per warp; the order of the list does not matter)
      const uint32_t vm = __ballot_sync(0xFFFFFFFFu, cand);
      if (vm) {
        uint32_t b0 = 0;
        if (lane == __ffs(vm) - 1) b0 = atomicAdd(&a.ctr->vis_count[bounce], (uint32_t)__popc(vm));
        b0 = __shfl_sync(0xFFFFFFFFu, b0, __ffs(vm) - 1);
        if (cand) {
          uint32_t cpos = vj_kid >= 0 ? kbase + (uint32_t)vj_kid : kNone;
          uint32_t rpos = vj_rec >= 0 ? rec0 + rbase + (uint32_t)vj_rec : kNone;
          if (cpos != kNone && cpos >= a.ray_cap) cpos = kNone;   // not written: the scan reports the overflow
          if (rpos != kNone && rpos >= a.rec_cap) rpos = kNone;
          VisJob* jw = reinterpret_cast<VisJob*>(a.rays[bounce & 1]) + i;
          jw->idx.y = cpos;
          jw->idx.z = rpos;
          a.vis_list[b0 + (uint32_t)__popc(vm & ((1u << lane) - 1u))] = i;
        }
      }
    }
    for (uint32_t c = 0; c < nk; ++c) {
      const uint32_t pos = kbase + c;
      if (pos < a.ray_cap) qout[pos] = kid[c];
    }
    if (a.order_key != nullptr && bounce + 1 < a.max_bounces) {
      // order buckets of the children, counted in the block's histogram
      for (uint32_t c = 0; c < nk; ++c) {
        const uint32_t pos = kbase + c;
        if (pos < a.ray_cap) {
          const uint32_t key = order_key(a, kid[c]);
          a.order_key[pos] = (uint16_t)key;
          atomicAdd(&s_hist[key], 1u);
        }
      }
    }
    for (uint32_t c = 0; c < nr; ++c) {
      const uint32_t pos = rec0 + rbase + c;
      if (pos < a.rec_cap) a.recs[pos] = rec[c];
    }
    if (tile == tiles - 1 && threadIdx.x == 0) {
      const uint32_t kids = ex.x + (total & 0xFFFFu), recs = ex.y + (total >> 16);
      ScanCounters* cn = a.ctr;
      uint32_t next = kids;
      if (kids > a.ray_cap) {
        atomicOr(&cn->error, kErrCapacityRays);
        atomicMax(&cn->need_rays, kids);
        next = a.ray_cap;
      }
      uint32_t rend = rec0 + recs;
      if (rend > a.rec_cap || rend < rec0) {
        atomicOr(&cn->error, kErrCapacityRecs);
        atomicMax(&cn->need_recs, rend);
        rend = a.rec_cap;
      }
      cn->count[bounce + 1] = next;   // rays past their scan's bounce limit spawn no children
      cn->rec_start[bounce + 1] = rend;
      cn->seg_start[bounce + 1] = seg0 + n;
      cn->stat_returns += (unsigned long long)recs;
    }
    __syncthreads();
  }
  // the block's bucket counts into the bounce's histogram (the loop ended
  // with a barrier, so every count is in)
  if (counting) {
    uint32_t* h = a.order_hist + (size_t)(bounce + 1) * kOrderBuckets;
    for (uint32_t j = threadIdx.x; j < kOrderBuckets; j += kShadeBlock)
      if (s_hist[j]) atomicAdd(&h[j], s_hist[j]);
  }
}

}  // namespace rr

namespace rr_host {

using namespace rr;

static int g_num_sms = 0;
static int g_query_occ[2][2][3] = {{{0}}};   // [wide][any][block 64 / 128 / 256]
static int g_shade_occ[2] = {0, 0};   // resident blocks of k_shade<3>, k_shade<4>

static int block_index(uint32_t block) { return block <= 64u ? 0 : (block <= 128u ? 1 : 2); }

template <bool kAny, int kBlock, bool kWide>
static void occ_of(int* out) {
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_query<kAny, kBlock, kWide, false>, kBlock, 0);
  if (*out < 1) *out = 1;
}

template <bool kWide>
static void occ_all(int (*o)[3]) {
  occ_of<false, 64, kWide>(&o[0][0]);
  occ_of<false, 128, kWide>(&o[0][1]);
  occ_of<false, 256, kWide>(&o[0][2]);
  occ_of<true, 64, kWide>(&o[1][0]);
  occ_of<true, 128, kWide>(&o[1][1]);
  occ_of<true, 256, kWide>(&o[1][2]);
}

void init_dims() {
  if (g_num_sms) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  occ_all<false>(g_query_occ[0]);
  occ_all<true>(g_query_occ[1]);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_shade_occ[0], k_shade<3>, kShadeBlock, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_shade_occ[1], k_shade<4>, kShadeBlock, 0);
  for (int& o : g_shade_occ)
    if (o < 1) o = 1;
  g_num_sms = sms < 1 ? 1 : sms;
}

int num_sms() {
  init_dims();
  return g_num_sms;
}

int trace_max_blocks_per_sm(uint32_t block, bool wide) {
  init_dims();
  return g_query_occ[wide ? 1 : 0][0][block_index(block)];
}

cudaError_t launch_raygen(const ScanArgs& a, cudaStream_t st) {
  const uint32_t n = a.n_rays0;
  k_raygen<<<n ? (n + 255) / 256 : 1, 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <bool kAny, bool kWide, bool kCount>
static void query_launch_c(const ScanArgs& a, uint32_t bounce, int bi, int grid, cudaStream_t st) {
  if (bi == 0) k_query<kAny, 64, kWide, kCount><<<grid, 64, 0, st>>>(a, bounce);
  else if (bi == 1) k_query<kAny, 128, kWide, kCount><<<grid, 128, 0, st>>>(a, bounce);
  else k_query<kAny, 256, kWide, kCount><<<grid, 256, 0, st>>>(a, bounce);
}
template <bool kAny, bool kWide>
static void query_launch(const ScanArgs& a, uint32_t bounce, int bi, int grid, cudaStream_t st) {
  // a counting kernel may hold more registers: its blocks beyond the
  // residency start later and find no work left
  if (a.any_flags & RR_COUNT_TRAVERSAL) query_launch_c<kAny, kWide, true>(a, bounce, bi, grid, st);
  else query_launch_c<kAny, kWide, false>(a, bounce, bi, grid, st);
}

cudaError_t launch_query(const ScanArgs& a, uint32_t bounce, bool any, const LaunchCfg& c, cudaStream_t st) {
  init_dims();
  const bool wide = a.wide != 0u;
  const int bi = block_index(c.trace_block);
  int per_sm = g_query_occ[wide ? 1 : 0][any ? 1 : 0][bi];
  if (c.trace_blocks_per_sm > 0 && (int)c.trace_blocks_per_sm < per_sm) per_sm = (int)c.trace_blocks_per_sm;
  const int grid = g_num_sms * per_sm;
  if (wide) {
    if (any) query_launch<true, true>(a, bounce, bi, grid, st);
    else query_launch<false, true>(a, bounce, bi, grid, st);
  } else {
    if (any) query_launch<true, false>(a, bounce, bi, grid, st);
    else query_launch<false, false>(a, bounce, bi, grid, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_vis_prep(const ScanArgs& a, uint32_t bounce, cudaStream_t st) {
  init_dims();
  k_vis_prep<<<g_num_sms * 8, 256, 0, st>>>(a, bounce);
  return cudaGetLastError();
}

cudaError_t launch_order(const ScanArgs& a, uint32_t bounce, cudaStream_t st) {
  init_dims();
  k_order_scan<<<1, 1024, 0, st>>>(a, bounce);
  k_order_place<<<g_num_sms * 4, 256, 0, st>>>(a, bounce);
  return cudaGetLastError();
}

cudaError_t launch_shade(const ScanArgs& a, uint32_t bounce, cudaStream_t st) {
  init_dims();
  const size_t smem = a.order_key ? kOrderBuckets * sizeof(uint32_t) : 0;
  if (a.n_rays0 >= kShadeManyRays)
    k_shade<4><<<g_num_sms * g_shade_occ[1], kShadeBlock, smem, st>>>(a, bounce);
  else
    k_shade<3><<<g_num_sms * g_shade_occ[0], kShadeBlock, smem, st>>>(a, bounce);
  return cudaGetLastError();
}

cudaError_t selftest_look_back_wait(void* scratch, cudaStream_t st, bool* gave_up) {
  // scratch: a zeroed ScanCounters, then two zeroed tile status words
  ScanArgs a;
  memset(&a, 0, sizeof a);
  a.ctr = static_cast<ScanCounters*>(scratch);
  a.tile_status = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + sizeof(ScanCounters));
  k_selftest_look_back<<<1, 32, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  uint32_t err = 0;
  e = cudaMemcpyAsync(&err, &a.ctr->error, sizeof err, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  *gave_up = (err & kErrTimeout) != 0u;
  return cudaSuccess;
}

}  // namespace rr_host
