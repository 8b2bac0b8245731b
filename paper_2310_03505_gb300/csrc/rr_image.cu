// rr_image.cu -- polar image assembly and post pass.
//
// Sec. III-B: every return lands in the pixel of its azimuth column and
// range bin; the pixel sums the energies from 0.  Sec. III-C: measurement
// noise as a Gaussian blur along range, a beam pattern across azimuths,
// additive uniform system and ambient noise.
//
// One CTA owns one image column (one azimuth of one scan of the batch; the
// batch's columns are numbered scan by scan): it finds the column's records in every
// bounce's record list (each list is in azimuth order, so two binary
// searches per bounce), accumulates them into a shared-memory histogram with
// warp-aggregated adds (lanes that hit the same bin are summed with shuffles
// and added once), blurs the column in shared memory, adds the noise and
// writes the column once, coalesced.  No global atomics, no memset.
//
// The sums are compensated (Neumaier's improvement of Kahan summation,
// ZAMM 54, 1974): every bin holds a float pair (sum, correction) updated with
// a 64-bit compare-and-swap, and lanes that share a bin combine their values
// the same way first, so a bin's error stays within a few units in the last
// place of its value however many returns it receives and in whatever order.
#include <cuda_runtime.h>

#include <cstring>

#include "rr_host.h"

namespace rr {

constexpr int kImgBlock = 256;
constexpr int kMaxTaps = 2 * 768 + 1;   // blur / pattern radius up to 768

__device__ __forceinline__ int gauss_taps(float sigma, float* w) {
  // normalised exp(-j^2 / (2 sigma^2)) for |j| <= ceil(3 sigma); w[0..2R]
  const int R = min((int)ceilf(3.0f * sigma), (kMaxTaps - 1) / 2);
  for (int j = threadIdx.x; j <= 2 * R; j += blockDim.x) {
    const float x = (float)(j - R) / sigma;
    w[j] = expf(-0.5f * x * x);
  }
  __syncthreads();
  __shared__ float s_norm;
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int j = 0; j <= 2 * R; ++j) s += w[j];
    s_norm = 1.0f / s;
  }
  __syncthreads();
  for (int j = threadIdx.x; j <= 2 * R; j += blockDim.x) w[j] *= s_norm;
  __syncthreads();
  return R;
}

// first record in [lo, hi) whose column is >= col (records are in column order)
__device__ __forceinline__ uint32_t lower_col(const uint2* __restrict__ recs, uint32_t lo, uint32_t hi, uint32_t col) {
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if ((__ldg(&recs[mid].x) >> kBinBits) < col) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Sec. III-C Perlin noise (Perlin, "Improving noise", SIGGRAPH 2002) of
// pixel (a, bin): gradient noise over a lattice of P = round(n_az / cell_az)
// cells around the circle (periodic) and cells of cell_bins bins along range;
// lattice point (I, J) has the unit gradient at angle 2 pi u, u the uniform of
// Philox counter (scan_id, I, J, purpose); quintic fade; value 1/2 + n/sqrt(2)
__device__ __forceinline__ float perlin_at(uint4 rng, uint32_t n_az, float cell_az, float cell_bins, uint32_t a,
                                          uint32_t bin, uint32_t purpose) {
  const int P = max(1, (int)roundf((float)n_az / cell_az));
  const float x = (float)a * (float)P / (float)n_az, y = (float)bin / cell_bins;
  const float xf = floorf(x), yf = floorf(y);
  const uint32_t i0 = (uint32_t)xf % (uint32_t)P, i1 = (i0 + 1u) % (uint32_t)P;
  const uint32_t j0 = (uint32_t)yf, j1 = j0 + 1u;
  const float fx = x - xf, fy = y - yf;
  float s00, c00, s10, c10, s01, c01, s11, c11;
  sincospif(2.0f * u01(draw(rng, i0, j0, purpose).x), &s00, &c00);
  sincospif(2.0f * u01(draw(rng, i1, j0, purpose).x), &s10, &c10);
  sincospif(2.0f * u01(draw(rng, i0, j1, purpose).x), &s01, &c01);
  sincospif(2.0f * u01(draw(rng, i1, j1, purpose).x), &s11, &c11);
  const float n00 = c00 * fx + s00 * fy, n10 = c10 * (fx - 1.0f) + s10 * fy;
  const float n01 = c01 * fx + s01 * (fy - 1.0f), n11 = c11 * (fx - 1.0f) + s11 * (fy - 1.0f);
  const float sx = fx * fx * fx * (fx * (6.0f * fx - 15.0f) + 10.0f);
  const float sy = fy * fy * fy * (fy * (6.0f * fy - 15.0f) + 10.0f);
  const float nx0 = n00 + sx * (n10 - n00), nx1 = n01 + sx * (n11 - n01);
  return 0.5f + (nx0 + sy * (nx1 - nx0)) * 0.70710678118654752f;
}

// Sec. III-C: system and ambient noise of one pixel, uniform or Perlin
__device__ __forceinline__ float noise_at(const ScanDesc* sd, uint4 rng, float4 post, uint32_t az, uint32_t bin) {
  if (rng.w & RR_NOISE_PERLIN) {
    const float4 ext = __ldg(&sd->ext);
    const uint32_t n_az = __ldg(&sd->dims.x);
    return post.z * perlin_at(rng, n_az, ext.y, ext.z, az, bin, 4u) +
           post.w * perlin_at(rng, n_az, ext.y, ext.z, az, bin, 5u);
  }
  return post.z * u01(draw(rng, az, bin, 2u).x) + post.w * u01(draw(rng, az, bin, 3u).x);
}

// (s, c) + (x, cx) with the rounding error of s + x carried into c
__device__ __forceinline__ float2 neumaier(float2 acc, float x, float cx) {
  const float t = acc.x + x;
  const float e = fabsf(acc.x) >= fabsf(x) ? (acc.x - t) + x : (x - t) + acc.x;
  return make_float2(t, acc.y + (e + cx));
}

__device__ __forceinline__ void bin_add(unsigned long long* cell, float x, float cx) {
  unsigned long long old = *cell, seen;
  do {
    seen = old;
    const float2 cur = make_float2(__uint_as_float((uint32_t)seen), __uint_as_float((uint32_t)(seen >> 32)));
    const float2 nxt = neumaier(cur, x, cx);
    const unsigned long long v = (unsigned long long)__float_as_uint(nxt.x) |
                                 ((unsigned long long)__float_as_uint(nxt.y) << 32);
    old = atomicCAS(cell, seen, v);
  } while (old != seen);
}

__global__ void __launch_bounds__(kImgBlock) k_bin_column(ScanArgs a) {
  extern __shared__ unsigned long long sm64[];
  unsigned long long* cells = sm64;                             // [n_bins] (sum, correction)
  float* hist = reinterpret_cast<float*>(sm64 + a.max_bins);    // [n_bins] the compensated sums
  float* col = reinterpret_cast<float*>(sm64);                  // [n_bins] after the blur (reuses cells)
  __shared__ float taps[kMaxTaps];
  __shared__ uint32_t s_rng[2 * RR_MAX_BOUNCES];
  const uint32_t c = blockIdx.x;
  const uint32_t scan = owner_of(a.col0, a.n_scans, c);
  const ScanDesc* sd = a.desc + scan;
  const uint32_t az = __ldg(&sd->offs.w) + (c - __ldg(&a.col0[scan]));   // the scan's first azimuth + column
  const uint32_t nb = __ldg(&sd->dims.w);
  const float4 post = __ldg(&sd->post);   // blur sigma, pattern sigma, noise_sys, noise_amb
  const int lane = threadIdx.x & 31;
  for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) cells[i] = 0ull;
  // record range of this column in every bounce's list: lane 2b / 2b+1
  if (threadIdx.x < 32) {
    const uint32_t b = (uint32_t)lane >> 1;
    if (b < a.max_bounces) {
      const uint32_t lo = a.ctr->rec_start[b], hi = a.ctr->rec_start[b + 1];
      s_rng[lane] = lower_col(a.recs, lo, hi, c + (lane & 1));
    }
  }
  __syncthreads();
  for (uint32_t b = 0; b < a.max_bounces; ++b) {
    const uint32_t lo = s_rng[2 * b], hi = s_rng[2 * b + 1];
    // whole warps iterate together so that the shuffles see every lane
    for (uint32_t base = lo; base < hi; base += blockDim.x) {
      const uint32_t r = base + threadIdx.x;
      bool valid = r < hi;
      uint32_t bin = 0;
      float e = 0.0f;
      if (valid) {
        const uint2 rc = __ldg(&a.recs[r]);
        bin = rc.x & kBinMask;
        e = __uint_as_float(rc.y);
        valid = bin < nb;   // records always carry bin < n_bins; a failed scan may leave stale slots
      }
      const uint32_t tag = valid ? bin : 0x10000u + (uint32_t)lane;
      const uint32_t peers = __match_any_sync(0xFFFFFFFFu, tag);
      float2 acc = make_float2(0.0f, 0.0f);
      for (uint32_t m = peers; m; m &= m - 1u) acc = neumaier(acc, __shfl_sync(peers, e, __ffs(m) - 1), 0.0f);
      if (valid && lane == __ffs(peers) - 1) bin_add(&cells[bin], acc.x, acc.y);
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) {
    const unsigned long long v = cells[i];
    hist[i] = __uint_as_float((uint32_t)v) + __uint_as_float((uint32_t)(v >> 32));
  }
  __syncthreads();
  const float* src = hist;
  if (post.x > 0.0f) {
    const int R = gauss_taps(post.x, taps);
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) {
      float acc = 0.0f;
      for (int j = -R; j <= R; ++j) {
        const int s = (int)i + j;
        if (s >= 0 && s < (int)nb) acc += taps[j + R] * hist[s];
      }
      col[i] = acc;
    }
    __syncthreads();
    src = col;
  }
  if (post.y > 0.0f) {
    float* out = a.image_tmp + __ldg(&sd->offs.z) + (size_t)az * nb;
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) out[i] = src[i];
  } else {
    float* out = sd->image + (size_t)az * nb;
    const uint4 rng = __ldg(&sd->rng);
    const bool noise = (rng.w & RR_NOISE) != 0u;
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x)
      out[i] = src[i] + (noise ? noise_at(sd, rng, post, az, i) : 0.0f);
  }
}

// beam pattern across the azimuths of a scan (circular), then noise; one
// block row per image column, scans without a pattern return at once
__global__ void __launch_bounds__(kImgBlock) k_az_pattern(ScanArgs a) {
  __shared__ float taps[kMaxTaps];
  const uint32_t c = blockIdx.x;   // column on x: a batch may hold more than 65535
  const uint32_t scan = owner_of(a.col0, a.n_scans, c);
  const ScanDesc* sd = a.desc + scan;
  const float4 post = __ldg(&sd->post);
  if (!(post.y > 0.0f)) return;   // uniform over the block
  const int R = gauss_taps(post.y, taps);
  const uint32_t az = __ldg(&sd->offs.w) + (c - __ldg(&a.col0[scan]));   // pattern scans are never split: offs.w = 0
  const uint32_t n_az = __ldg(&sd->dims.x), nb = __ldg(&sd->dims.w);
  const uint32_t i = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const float* tmp = a.image_tmp + __ldg(&sd->offs.z);
  float acc = 0.0f;
  for (int j = -R; j <= R; ++j) {
    int s = ((int)az + j) % (int)n_az;
    if (s < 0) s += (int)n_az;
    acc += taps[j + R] * tmp[(size_t)s * nb + i];
  }
  const uint4 rng = __ldg(&sd->rng);
  if (rng.w & RR_NOISE) acc += noise_at(sd, rng, post, az, i);
  sd->image[(size_t)az * nb + i] = acc;
}

// records of caller-given returns: (column << kBinBits | bin, energy); flags
// a column that decreases or lies past the image
__global__ void k_pack_returns(const uint32_t* __restrict__ column, const uint32_t* __restrict__ bin,
                               const float* __restrict__ energy, uint32_t n, uint32_t n_columns, uint32_t n_bins,
                               uint2* __restrict__ recs, uint32_t* __restrict__ bad) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t c = column[k], b = bin[k];
  if ((k > 0 && column[k - 1] > c) || c >= n_columns) atomicOr(bad, 1u);
  // a bin past the image contributes nothing
  const bool in = b < n_bins;
  recs[k] = make_uint2(((c < n_columns ? c : 0u) << kBinBits) | (in ? b : 0u), in ? __float_as_uint(energy[k]) : 0u);
}

// Sec. III-B display mapping
__global__ void k_db_u8(const float* __restrict__ polar, uint64_t n, float cutoff_db, uint8_t* __restrict__ out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float e = polar[i];
  float v = 0.0f;
  if (e > 0.0f) v = fminf(fmaxf(255.0f * (10.0f * log10f(e) + cutoff_db) / cutoff_db, 0.0f), 255.0f);
  out[i] = (uint8_t)floorf(v + 0.5f);
}

}  // namespace rr

namespace rr_host {

using namespace rr;

// dynamic shared memory of k_bin_column: (sum, correction) pairs (later the
// blurred column), sums
static size_t bin_smem(uint32_t n_bins) { return (size_t)n_bins * (sizeof(unsigned long long) + sizeof(float)); }

void init_image_attrs() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_bin_column, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bin_smem(RR_MAX_BINS));
    attr_set = true;
  }
}

cudaError_t launch_image(const ScanArgs& a, bool pattern, cudaStream_t st) {
  init_image_attrs();
  k_bin_column<<<a.n_cols, kImgBlock, bin_smem(a.max_bins), st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (pattern) {
    dim3 grid(a.n_cols, (a.max_bins + kImgBlock - 1) / kImgBlock);
    k_az_pattern<<<grid, kImgBlock, 0, st>>>(a);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_db_u8(const float* polar, uint64_t n, float cutoff_db, uint8_t* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_db_u8<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(polar, n, cutoff_db, out);
  return cudaGetLastError();
}

}  // namespace rr_host

using namespace rr_host;

extern "C" int rr_accumulate_returns(const uint32_t* column, const uint32_t* bin, const float* energy, uint64_t n,
                                     uint32_t n_columns, uint32_t n_bins, float* out) {
  if (!out || (n && (!column || !bin || !energy))) return fail(RR_ERR_INVALID_ARG, "NULL buffer");
  if (n_columns < 1 || n_columns > kMaxColumns) return fail(RR_ERR_INVALID_ARG, "n_columns must be in [1, 2^18]");
  if (n_bins < 1 || n_bins > RR_MAX_BINS) return fail(RR_ERR_INVALID_ARG, "n_bins must be in [1, 16384]");
  if (n >= (1ull << 31)) return fail(RR_ERR_INVALID_ARG, "at most 2^31 - 1 returns");
  cudaStream_t st = current_stream();
  const size_t img_bytes = (size_t)n_columns * n_bins * sizeof(float);
  // device scratch of this call: inputs, records, a counter block, one scan
  // descriptor with its prefix arrays, the image
  uint32_t *d_col = nullptr, *d_bin = nullptr, *d_bad = nullptr;
  float *d_e = nullptr, *d_img = nullptr;
  uint2* d_recs = nullptr;
  ScanCounters* d_ctr = nullptr;
  ScanDesc* d_desc = nullptr;
  uint32_t* d_pre = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    for (void* p : {(void*)d_col, (void*)d_bin, (void*)d_bad, (void*)d_e, (void*)d_img, (void*)d_recs, (void*)d_ctr,
                    (void*)d_desc, (void*)d_pre})
      if (p) cudaFree(p);
  };
  cudaError_t e = cudaSuccess;
  const size_t nn = n ? n : 1;
  if (e == cudaSuccess) e = dev_malloc(&d_col, nn * 4);
  if (e == cudaSuccess) e = dev_malloc(&d_bin, nn * 4);
  if (e == cudaSuccess) e = dev_malloc(&d_e, nn * 4);
  if (e == cudaSuccess) e = dev_malloc(&d_recs, nn * 8);
  if (e == cudaSuccess) e = dev_malloc(&d_bad, 4);
  if (e == cudaSuccess) e = dev_malloc(&d_img, img_bytes);
  if (e == cudaSuccess) e = dev_malloc(&d_ctr, sizeof(ScanCounters));
  if (e == cudaSuccess) e = dev_malloc(&d_desc, sizeof(ScanDesc));
  if (e == cudaSuccess) e = dev_malloc(&d_pre, 4 * sizeof(uint32_t));
  if (e == cudaSuccess && n) e = cudaMemcpyAsync(d_col, column, n * 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess && n) e = cudaMemcpyAsync(d_bin, bin, n * 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess && n) e = cudaMemcpyAsync(d_e, energy, n * 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_ctr, 0, sizeof(ScanCounters), st);
  ScanDesc desc;
  memset(&desc, 0, sizeof desc);
  desc.dims = make_uint4(n_columns, 1u, 1u, n_bins);
  desc.offs = make_uint4(0u, 0u, kNone, 0u);
  desc.image = d_img;
  const uint32_t pre[4] = {0u, 0u, 0u, n_columns};   // ray prefix (unused) and column prefix
  const uint32_t starts[2] = {0u, (uint32_t)n};
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_desc, &desc, sizeof desc, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_pre, pre, sizeof pre, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&d_ctr->rec_start[0], starts, sizeof starts, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n) {
    k_pack_returns<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_col, d_bin, d_e, (uint32_t)n, n_columns, n_bins,
                                                                 d_recs, d_bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host copies above came from the stack
  uint32_t bad = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&bad, d_bad, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return cuda_fail(e, "accumulating the returns");
  }
  if (bad) {
    cleanup();
    return fail(RR_ERR_INVALID_ARG, "column must be non-decreasing and below n_columns");
  }
  ScanArgs a;
  memset(&a, 0, sizeof a);
  a.desc = d_desc;
  a.ray0 = d_pre;
  a.col0 = d_pre + 2;
  a.n_scans = 1;
  a.n_cols = n_columns;
  a.max_bounces = 1;
  a.max_bins = n_bins;
  a.recs = d_recs;
  a.ctr = d_ctr;
  a.rec_cap = (uint32_t)nn;
  e = launch_image(a, false, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_img, img_bytes, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return cuda_fail(e, "accumulating the returns");
  }
  cleanup();
  return RR_OK;
}
