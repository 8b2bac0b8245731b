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
#include <cuda_runtime.h>

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

// Sec. III-C: uniform system and ambient noise of one pixel
__device__ __forceinline__ float noise_at(uint4 rng, float4 post, uint32_t az, uint32_t bin) {
  return post.z * u01(draw(rng, az, bin, 2u).x) + post.w * u01(draw(rng, az, bin, 3u).x);
}

__global__ void __launch_bounds__(kImgBlock) k_bin_column(ScanArgs a) {
  extern __shared__ float sm[];
  float* hist = sm;                     // [n_bins]
  float* col = sm + a.max_bins;         // [n_bins]
  __shared__ float taps[kMaxTaps];
  __shared__ uint32_t s_rng[2 * RR_MAX_BOUNCES];
  const uint32_t c = blockIdx.x;
  const uint32_t scan = owner_of(a.col0, a.n_scans, c);
  const ScanDesc* sd = a.desc + scan;
  const uint32_t az = c - __ldg(&a.col0[scan]);
  const uint32_t nb = __ldg(&sd->dims.w);
  const float4 post = __ldg(&sd->post);   // blur sigma, pattern sigma, noise_sys, noise_amb
  const int lane = threadIdx.x & 31;
  for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0.0f;
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
      float sum = 0.0f;
      for (uint32_t m = peers; m; m &= m - 1u) sum += __shfl_sync(peers, e, __ffs(m) - 1);
      if (valid && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], sum);
    }
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
      out[i] = src[i] + (noise ? noise_at(rng, post, az, i) : 0.0f);
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
  const uint32_t az = c - __ldg(&a.col0[scan]);
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
  if (rng.w & RR_NOISE) acc += noise_at(rng, post, az, i);
  sd->image[(size_t)az * nb + i] = acc;
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

void init_image_attrs() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_bin_column, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * RR_MAX_BINS * (int)sizeof(float));
    attr_set = true;
  }
}

cudaError_t launch_image(const ScanArgs& a, bool pattern, cudaStream_t st) {
  init_image_attrs();
  const size_t smem = 2 * (size_t)a.max_bins * sizeof(float);
  k_bin_column<<<a.n_cols, kImgBlock, smem, st>>>(a);
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
