/*
 * rr_oracle.c -- FP64 brute-force CPU oracle of the RadaRays polar scan.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check of the package entry
 * module and the CPU-baseline leg of the benchmark are the only callers.  The
 * CUDA library never links, loads or calls this file, and this file shares no
 * code, header, table or constant generator with it: every formula is written
 * again here from the paper (Mock, Magnusson, Hertzberg: "RadaRays: Real-time
 * Simulation of Rotating FMCW Radar for Mobile Robotics via Hardware-accelerated
 * Ray Tracing", arXiv 2310.03505).
 *
 * Plain and slow on purpose:
 *   - every quantity is a double;
 *   - the closest hit is a loop over every triangle (Moller-Trumbore), no BVH
 *     (orc_scan; orc_scan_accel answers the same queries through a CPU BVH
 *     for the timed CPU baseline, pinned to give the same segments, flags,
 *     tallies and images as the loops);
 *   - each initial ray's tree is expanded depth first with an explicit stack;
 *   - returns are collected in a list and then summed into the polar image by
 *     a lookup, as Sec. III-B describes.
 *
 * Readings of passages the paper leaves open are fixed once here and listed in
 * the design notes of the repository (normalised Eq. 5, unpolarised Fresnel,
 * optical range, returns deplete the reflected child, air-path capping, ...).
 *
 * Parity flags.  Besides the image, the oracle marks every initial ray whose
 * tree contains a decision that FP32 arithmetic could take the other way
 * (a hit or a near miss within 1e-5 barycentric margin of a triangle edge,
 * a hit next to t_min or the range limit, a near tie between two triangles,
 * a total-internal-reflection test next to the critical angle, a refraction
 * so close to grazing that Snell's law amplifies rounding, a grazing hit, a
 * child next to the range cut).  Returns whose range sits next to a bin edge
 * add their energy to a per-bin slack.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NONE 0xFFFFFFFFu
#define ORC_AIR (-1)

#define ORC_MULTIPATH 1u
#define ORC_REFRACTION 2u
#define ORC_SPECKLE 4u
#define ORC_NOISE 8u
#define ORC_NOISE_PERLIN 32u

/* flag thresholds of the parity protocol */
#define FLAG_BARY 1e-5    /* barycentric margin (hits and near misses)        */
#define FLAG_TREL 1e-6    /* relative distance for ties / range limits        */
#define FLAG_TABS 1e-6    /* absolute distance next to t_min (metres)          */
#define FLAG_TIR 1e-6     /* |eta^2 sin^2 - 1| next to the critical angle      */
#define FLAG_COS 1e-6     /* grazing incidence |cos theta0|                    */
#define FLAG_EMAX 1e-2    /* largest edge distance (m) a hit point's error    */
                          /* estimate flags; above it the segment is flagged */
                          /* outright (the CPU BVH's boxes are grown by more */
                          /* than this)                                      */
#define FLAG_TDIR 1e-5    /* angle error (rad) of a refracted direction: the  */
                          /* relative hit-distance tolerance of the parity   */
#define FLAG_TALLY 8e-6   /* energy a tally may move by, relative to the      */
                          /* initial ray's energy (half its tolerance)       */

/* segment flag bits (diagnostics) */
#define SEG_EDGE 1u
#define SEG_TMIN 2u
#define SEG_TIE 4u
#define SEG_TLIM 8u
#define SEG_TIR 16u
#define SEG_GRAZE 32u
#define SEG_RMAX 64u
#define SEG_VIS 128u
#define SEG_EMIN 256u
#define SEG_SNELL 512u
#define SEG_TALLY 1024u   /* affects only the per-ray energy tallies */
#define SEG_ERR 2048u     /* FLAG_SIGMAS times a hit point's float32 error exceeds FLAG_EMAX */

/* lobe kinds of a material (Sec. III-A: user-defined BRDFs per material) */
#define ORC_LOBE_EQ5 0           /* Eq. 5 with A, B, C                                  */
#define ORC_LOBE_COOK_TORRANCE 1 /* microfacet lobe, A = diffuse amount, B = roughness  */
#define ORC_LOBE_TABLE 2         /* tabulated density, table[ORC_LOBE_SAMPLES]          */
#define ORC_LOBE_CELLS 2048
#define ORC_LOBE_SAMPLES (2 * ORC_LOBE_CELLS + 1)

typedef struct {
  double eps_r, loss_tangent, A, B, C;
  int32_t pec, lobe;
  const double* table; /* ORC_LOBE_TABLE: density at x_j = j (pi/2) / (2 ORC_LOBE_CELLS) */
} orc_material;

typedef struct {
  uint32_t n_azimuth, rays_per_beam, max_bounces, n_bins;
  double beam_width, beam_prob, elevation, bin_size, t_min, min_energy, freq_hz;
  double blur_sigma_bins, az_pattern_sigma, noise_sys, noise_amb;
  uint32_t flags, seed_lo, seed_hi, scan_id;
  double beam_aspect;                   /* elevation / azimuth spread of the D3 cone (1: circular) */
  double noise_cell_az, noise_cell_bins; /* Perlin lattice spacing (beams, bins) */
  uint32_t ray_stride;                  /* trace the initial rays k = 0, s, 2s, ... of each column (0, 1: all);
                                           a sample: each ray is independent of the others */
  double range_falloff;                 /* exponent k of the optional range weight (1 m / r)^k of a
                                           return at range r > 1 m (Eq. 1's R^-4 with k = 4; 0: off) */
} orc_params;

typedef struct {
  double p[3];
  double q[4]; /* (w, x, y, z) */
} orc_pose;

typedef struct {
  uint32_t az, k, path, bounce, tri, flags;
  double t, E;
  double cos_i, ret_t, ret_a;
  double e_org, e_dir; /* float32 error estimate (standard deviations) of the segment's origin (m, moved
                          within the hit plane it starts on: the distance tolerances) and direction (rad) */
  double alpha2;       /* power attenuation constant 2 alpha (1/m) of the medium the segment crosses (0: air) */
} orc_segment;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC 2011).  Ten rounds of two 32x32->64 multiplications  */
/* with a Weyl-sequence key schedule.                                       */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint64_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
  const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = mul0 * (uint64_t)c0;
    uint64_t prod1 = mul1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += weyl0;
    k1 += weyl1;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* uniform in (0,1) from the top 23 bits: (2 (x >> 9) + 1) / 2^24.  The odd
   numerator has at most 24 significant bits, so the value is exact in float
   as well as in double and both implementations draw identical numbers. */
double orc_u24(uint32_t x) { return (double)(2u * (x >> 9) + 1u) * (1.0 / 16777216.0); }

static void draw(const orc_params* p, uint32_t a, uint32_t b, uint32_t c, uint32_t out[4]) {
  uint32_t ctr[4] = {p->scan_id, a, b, c};
  uint32_t key[2] = {p->seed_lo, p->seed_hi};
  orc_philox(ctr, key, out);
}

/* inverse error function: bisection on erf() to full double precision */
double orc_erfinv(double y) {
  if (!(y > -1.0 && y < 1.0)) return NAN;
  double lo = -6.0, hi = 6.0;
  for (int i = 0; i < 200; ++i) {
    double mid = 0.5 * (lo + hi);
    if (erf(mid) < y) lo = mid; else hi = mid;
    if (hi - lo <= 0.0) break;
  }
  return 0.5 * (lo + hi);
}

/* Eq. 2: standard deviation of the D3 radius, sigma = (b/2) / (sqrt(2) erfinv(P)) */
double orc_d3_sigma(double beam_width, double beam_prob) {
  if (beam_width == 0.0) return 0.0;
  return 0.5 * beam_width / (sqrt(2.0) * orc_erfinv(beam_prob));
}

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                     */
/* ------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static void sub3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[0] - b[0];
  o[1] = a[1] - b[1];
  o[2] = a[2] - b[2];
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static void normalize3(double a[3]) {
  double n = norm3(a);
  a[0] /= n;
  a[1] /= n;
  a[2] /= n;
}
/* angle between two vectors, atan2(|a x b|, a.b) */
double orc_angle(const double a[3], const double b[3]) {
  double c[3];
  cross3(a, b, c);
  return atan2(norm3(c), dot3(a, b));
}

/* rotate v by the unit quaternion q = (w, x, y, z), written as its rotation matrix */
static void quat_rotate(const double qin[4], const double v[3], double o[3]) {
  double n = sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
  double w = qin[0] / n, x = qin[1] / n, y = qin[2] / n, z = qin[3] / n;
  double m[3][3] = {
      {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
      {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
      {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
  for (int i = 0; i < 3; ++i) o[i] = m[i][0] * v[0] + m[i][1] * v[1] + m[i][2] * v[2];
}

/* beam axis of azimuth index a in the world frame */
void orc_beam_axis(const orc_params* p, const orc_pose* pose, uint32_t a, double axis[3]) {
  double phi = 2.0 * M_PI * (double)a / (double)p->n_azimuth;
  double th = p->elevation;
  double ds[3] = {cos(th) * cos(phi), cos(th) * sin(phi), sin(th)};
  quat_rotate(pose->q, ds, axis);
}

/* ------------------------------------------------------------------------ */
/* Sec. III-A, Eq. 2: D3 cone sample of initial ray k of azimuth a.          */
/* N ~ N(0,1) by Box-Muller from two uniforms, omega ~ U[-pi, pi), r = sigma N */
/* (d_az, d_inc) = r (cos omega, a sin omega) around the beam axis: a = 1 is */
/* the circular cone, a != 1 the cone stretched along the elevation axis     */
/* (elliptic beams, Sec. III-A).                                             */
/* ------------------------------------------------------------------------ */
void orc_d3_ray(const orc_params* p, const orc_pose* pose, uint32_t a, uint32_t k, double o[3], double d[3],
                double* r_out, double* omega_out) {
  uint32_t x[4];
  draw(p, a, k, 0u, x);
  double u0 = orc_u24(x[0]), u1 = orc_u24(x[1]), u2 = orc_u24(x[2]);
  double gauss = sqrt(-2.0 * log(u0)) * cos(2.0 * M_PI * u1);
  double sigma = orc_d3_sigma(p->beam_width, p->beam_prob);
  double r = sigma * gauss;
  double omega = M_PI * (2.0 * u2 - 1.0);
  double phi = 2.0 * M_PI * (double)a / (double)p->n_azimuth + r * cos(omega);
  double th = p->elevation + p->beam_aspect * r * sin(omega);
  double ds[3] = {cos(th) * cos(phi), cos(th) * sin(phi), sin(th)};
  quat_rotate(pose->q, ds, d);
  normalize3(d);
  o[0] = pose->p[0];
  o[1] = pose->p[1];
  o[2] = pose->p[2];
  if (r_out) *r_out = r;
  if (omega_out) *omega_out = omega;
}

/* ------------------------------------------------------------------------ */
/* Sec. III-A: Fresnel split of the incident energy E0 = E1 + E2 and Snell's */
/* law sin(theta0)/sin(theta2) = v1/v2 = n2/n1.  Unpolarised: R = (Rs+Rp)/2. */
/* Returns 1 on total internal reflection (R = 1, T = 0).                    */
/* ------------------------------------------------------------------------ */
int orc_fresnel(double n1, double n2, double cos_i, double* R, double* cos_t, double* sin2_t_out) {
  double eta = n1 / n2;
  double sin2_t = eta * eta * (1.0 - cos_i * cos_i);
  if (sin2_t_out) *sin2_t_out = sin2_t;
  if (sin2_t >= 1.0) {
    *R = 1.0;
    *cos_t = 0.0;
    return 1;
  }
  double ct = sqrt(1.0 - sin2_t);
  double rs = (n1 * cos_i - n2 * ct) / (n1 * cos_i + n2 * ct);
  double rp = (n1 * ct - n2 * cos_i) / (n1 * ct + n2 * cos_i);
  *R = 0.5 * (rs * rs + rp * rp);
  *cos_t = ct;
  return 0;
}

/* mirror direction about a unit normal n (theta1 = theta0) */
void orc_reflect(const double d[3], const double n[3], double out[3]) {
  double dn = dot3(d, n);
  for (int i = 0; i < 3; ++i) out[i] = d[i] - 2.0 * dn * n[i];
}

/* refracted direction; n faces the incident side (d.n = -cos_i < 0), eta = n1/n2 */
void orc_refract(const double d[3], const double n[3], double eta, double cos_i, double cos_t, double out[3]) {
  for (int i = 0; i < 3; ++i) out[i] = eta * d[i] + (eta * cos_i - cos_t) * n[i];
}

/* ------------------------------------------------------------------------ */
/* Eq. 3 - Eq. 5: BRDF lobe f(w) = (A + B cos w + S cos^C w) / Z on          */
/* [-pi/2, pi/2], S = 1 - A - B, normalised so that its integral is one,     */
/* and the beam-window fraction W(w) = integral of f over [w-b/2, w+b/2].    */
/* ------------------------------------------------------------------------ */
static double cospow(double x, double c) {
  double cx = cos(x);
  if (cx <= 0.0) return (c == 0.0) ? 1.0 : 0.0;
  return pow(cx, c);
}

static double simpson_rec(double c, double a, double b, double fa, double fm, double fb, double whole, double eps,
                          int depth) {
  double m = 0.5 * (a + b);
  double lm = 0.5 * (a + m), rm = 0.5 * (m + b);
  double flm = cospow(lm, c), frm = cospow(rm, c);
  double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
  double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
  double delta = left + right - whole;
  if (depth <= 0 || fabs(delta) <= 15.0 * eps) return left + right + delta / 15.0;
  return simpson_rec(c, a, m, fa, flm, fm, left, 0.5 * eps, depth - 1) +
         simpson_rec(c, m, b, fm, frm, fb, right, 0.5 * eps, depth - 1);
}

/* integral of cos^C over [lo, hi] by adaptive Simpson on 64 starting panels */
double orc_int_cospow(double c, double lo, double hi) {
  if (!(hi > lo)) return 0.0;
  const int panels = 64;
  double h = (hi - lo) / panels, sum = 0.0;
  for (int i = 0; i < panels; ++i) {
    double a = lo + h * i, b = (i == panels - 1) ? hi : lo + h * (i + 1);
    double fa = cospow(a, c), fb = cospow(b, c), fm = cospow(0.5 * (a + b), c);
    double whole = (b - a) / 6.0 * (fa + 4.0 * fm + fb);
    sum += simpson_rec(c, a, b, fa, fm, fb, whole, 1e-16, 48);
  }
  return sum;
}

/* ------------------------------------------------------------------------ */
/* Cook-Torrance lobe (the microfacet model the paper uses as a user BRDF,   */
/* Sec. IV; Cook & Torrance 1982, Walter et al. 2007).  Read on the same     */
/* 1-D domain as Eq. 5: w is the deviation of the return from the mirror     */
/* direction, whose half vector deviates from the normal by w/2.  The lobe  */
/* is a diffuse part cos(w)/2 plus a Beckmann microfacet part, each of unit  */
/* integral over [-pi/2, pi/2]:                                              */
/*   f(w) = kd cos(w)/2 + (1 - kd) D(w/2) / Zw,                              */
/*   D(t) = exp(-tan^2 t / m^2) / (pi m^2 cos^4 t),  kd = A, m = B,          */
/*   Zw = integral of D(w/2) over [-pi/2, pi/2] = 2 integral of D over       */
/*        [-pi/4, pi/4] = 2 [m sqrt(pi) erf(1/m) (1 + m^2/2) - m^2 e^(-1/m^2)] */
/*        / (pi m^2)   (substituting u = tan t).                             */
/* ------------------------------------------------------------------------ */
double orc_beckmann(double t, double m) {
  double c = cos(t), tt = tan(t);
  return exp(-tt * tt / (m * m)) / (M_PI * m * m * c * c * c * c);
}

double orc_beckmann_norm(double m) {
  return 2.0 * (m * sqrt(M_PI) * erf(1.0 / m) * (1.0 + 0.5 * m * m) - m * m * exp(-1.0 / (m * m))) / (M_PI * m * m);
}

static double ct_density(const orc_material* m, double w) {
  return m->A * 0.5 * cos(w) + (1.0 - m->A) * orc_beckmann(0.5 * w, m->B) / orc_beckmann_norm(m->B);
}

/* adaptive Simpson of the Cook-Torrance density over [a, b] */
static double ct_rec(const orc_material* m, double a, double b, double fa, double fm, double fb, double whole,
                     double eps, int depth) {
  double c = 0.5 * (a + b), lm = 0.5 * (a + c), rm = 0.5 * (c + b);
  double flm = ct_density(m, lm), frm = ct_density(m, rm);
  double left = (c - a) / 6.0 * (fa + 4.0 * flm + fm), right = (b - c) / 6.0 * (fm + 4.0 * frm + fb);
  double delta = left + right - whole;
  if (depth <= 0 || fabs(delta) <= 15.0 * eps) return left + right + delta / 15.0;
  return ct_rec(m, a, c, fa, flm, fm, left, 0.5 * eps, depth - 1) +
         ct_rec(m, c, b, fm, frm, fb, right, 0.5 * eps, depth - 1);
}

static double ct_integral(const orc_material* m, double lo, double hi) {
  const int panels = 256;
  double h = (hi - lo) / panels, sum = 0.0;
  for (int i = 0; i < panels; ++i) {
    double a = lo + h * i, b = (i == panels - 1) ? hi : lo + h * (i + 1);
    double fa = ct_density(m, a), fb = ct_density(m, b), fm = ct_density(m, 0.5 * (a + b));
    sum += ct_rec(m, a, b, fa, fm, fb, (b - a) / 6.0 * (fa + 4.0 * fm + fb), 1e-17, 48);
  }
  return sum;
}

/* ------------------------------------------------------------------------ */
/* Tabulated lobe (Sec. III-A: a user-defined BRDF per material): a          */
/* symmetric density given at x_j = j h, h = (pi/2) / (2 ORC_LOBE_CELLS),    */
/* read as the quadratic through (x_2k, x_2k+1, x_2k+2) on every cell, so    */
/* that Simpson's rule integrates each cell exactly.  Normalised to unit     */
/* integral over [-pi/2, pi/2].                                              */
/* ------------------------------------------------------------------------ */
/* integral of cell k's quadratic from its start to local coordinate s in [0, 2] (units of h) */
static double table_cell_prim(const double* t, int k, double s) {
  double f0 = t[2 * k], f1 = t[2 * k + 1], f2 = t[2 * k + 2];
  double s2 = s * s, s3 = s2 * s;
  return f0 * (s3 / 6.0 - 0.75 * s2 + s) - f1 * (s3 / 3.0 - s2) + f2 * (s3 / 6.0 - 0.25 * s2);
}

/* integral of the tabulated density over [0, x], 0 <= x <= pi/2 */
static double table_prim(const double* t, double x) {
  const double h = 0.5 * M_PI / (2.0 * ORC_LOBE_CELLS);
  double u = x / (2.0 * h);   /* in cells */
  if (u <= 0.0) return 0.0;
  if (u > ORC_LOBE_CELLS) u = ORC_LOBE_CELLS;
  int k = (int)floor(u);
  if (k >= ORC_LOBE_CELLS) k = ORC_LOBE_CELLS - 1;
  double sum = 0.0;
  for (int c = 0; c < k; ++c) sum += table_cell_prim(t, c, 2.0);
  sum += table_cell_prim(t, k, 2.0 * (u - k));
  return h * sum;
}

static double table_value(const double* t, double x) {
  const double h = 0.5 * M_PI / (2.0 * ORC_LOBE_CELLS);
  x = fabs(x);
  double u = x / (2.0 * h);
  int k = (int)floor(u);
  if (k >= ORC_LOBE_CELLS) k = ORC_LOBE_CELLS - 1;
  double s = 2.0 * (u - k);
  double f0 = t[2 * k], f1 = t[2 * k + 1], f2 = t[2 * k + 2];
  return f0 * (s - 1.0) * (s - 2.0) * 0.5 - f1 * s * (s - 2.0) + f2 * s * (s - 1.0) * 0.5;
}

/* signed-range integral of the symmetric tabulated density over [lo, hi] */
static double table_integral(const double* t, double lo, double hi) {
  if (lo >= 0.0) return table_prim(t, hi) - table_prim(t, lo);
  if (hi <= 0.0) return table_prim(t, -lo) - table_prim(t, -hi);
  return table_prim(t, hi) + table_prim(t, -lo);
}

/* Z = A pi + 2 B + S sqrt(pi) Gamma((C+1)/2) / Gamma(C/2 + 1) for Eq. 5;
   the integral of the density over [-pi/2, pi/2] for the other lobes */
double orc_brdf_norm(const orc_material* m) {
  if (m->lobe == ORC_LOBE_COOK_TORRANCE) return 1.0;
  if (m->lobe == ORC_LOBE_TABLE) return 2.0 * table_prim(m->table, M_PI / 2);
  double S = 1.0 - m->A - m->B;
  double gr = exp(lgamma(0.5 * (m->C + 1.0)) - lgamma(0.5 * m->C + 1.0));
  return m->A * M_PI + 2.0 * m->B + S * sqrt(M_PI) * gr;
}

double orc_brdf_density(const orc_material* m, double w) {
  if (w < -M_PI / 2 || w > M_PI / 2) return 0.0;
  if (m->lobe == ORC_LOBE_COOK_TORRANCE) return ct_density(m, w);
  if (m->lobe == ORC_LOBE_TABLE) return table_value(m->table, w) / orc_brdf_norm(m);
  double S = 1.0 - m->A - m->B;
  return (m->A + m->B * cos(w) + S * cospow(w, m->C)) / orc_brdf_norm(m);
}

double orc_brdf_window(const orc_material* m, double w, double b) {
  double lo = w - 0.5 * b, hi = w + 0.5 * b;
  if (lo < -M_PI / 2) lo = -M_PI / 2;
  if (hi > M_PI / 2) hi = M_PI / 2;
  if (!(hi > lo)) return 0.0;
  if (m->lobe == ORC_LOBE_COOK_TORRANCE) return ct_integral(m, lo, hi);
  if (m->lobe == ORC_LOBE_TABLE) return table_integral(m->table, lo, hi) / orc_brdf_norm(m);
  double S = 1.0 - m->A - m->B;
  double v = m->A * (hi - lo) + m->B * (sin(hi) - sin(lo));
  if (S != 0.0) v += S * orc_int_cospow(m->C, lo, hi);
  return v / orc_brdf_norm(m);
}

/* ------------------------------------------------------------------------ */
/* Moller-Trumbore ray/triangle test in double precision.  Reports the plane  */
/* distance t and the signed barycentrics (b1 for v1, b2 for v2) even when   */
/* the point lies outside, so the caller can see near misses.  Returns 0 if */
/* the ray is parallel to the plane.                                         */
/* ------------------------------------------------------------------------ */
int orc_tri_plane(const double o[3], const double d[3], const double v0[3], const double v1[3], const double v2[3],
                  double* t, double* b1, double* b2) {
  double e1[3], e2[3], pv[3], tv[3], qv[3];
  sub3(v1, v0, e1);
  sub3(v2, v0, e2);
  cross3(d, e2, pv);
  double det = dot3(e1, pv);
  if (det == 0.0) return 0;
  double inv = 1.0 / det;
  sub3(o, v0, tv);
  *b1 = dot3(tv, pv) * inv;
  cross3(tv, e1, qv);
  *b2 = dot3(d, qv) * inv;
  *t = dot3(e2, qv) * inv;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* scene                                                                    */
/* ------------------------------------------------------------------------ */
typedef struct orc_bvh orc_bvh;

typedef struct {
  const float* vtx;
  const uint32_t* tri;
  const uint16_t* mat_id;
  const orc_material* mat;
  uint32_t nv, nt, nm;
  const orc_bvh* bvh; /* NULL: brute force over all triangles (the oracle) */
  int fast;           /* with a BVH: no parity flags, strict pruning, tabulated windows */
} scene_t;

static void tri_vertices(const scene_t* s, uint32_t j, double v0[3], double v1[3], double v2[3]) {
  const uint32_t* t = s->tri + 3 * (size_t)j;
  for (int i = 0; i < 3; ++i) {
    v0[i] = (double)s->vtx[3 * (size_t)t[0] + i];
    v1[i] = (double)s->vtx[3 * (size_t)t[1] + i];
    v2[i] = (double)s->vtx[3 * (size_t)t[2] + i];
  }
}

/* geometric normal normalize((v1 - v0) x (v2 - v0)); triangles are wound so it
   points out of their material */
static void tri_normal(const scene_t* s, uint32_t j, double n[3]) {
  double v0[3], v1[3], v2[3], e1[3], e2[3];
  tri_vertices(s, j, v0, v1, v2);
  sub3(v1, v0, e1);
  sub3(v2, v0, e2);
  cross3(e1, e2, n);
  normalize3(n);
}

/* ------------------------------------------------------------------------ */
/* Float32 error estimate.  The CUDA path holds ray origins, directions and */
/* hit points in float32, so its hit points drift from this oracle's by an  */
/* amount that grows along the path.  Each rounding moves a value by a      */
/* uniform fraction of half an ulp (standard deviation 0.29 ulp); the many  */
/* independent roundings along a path add up like a random walk, so each   */
/* ray carries standard deviations: e_org (m) of its origin and e_dir (rad) */
/* of its direction, combined in quadrature.  Ray generation starts at      */
/* e_org = 0 (the pose position is a float) and e_dir = ERR_DIR0 ulps (the  */
/* beam angle, the angle sum, the elevation, the pose rotation and the      */
/* normalisation: about a dozen roundings); the hit point at distance t     */
/* adds t e_dir, half an ulp of its largest coordinate (the rounding of     */
/* o + t d) and one ulp of t (the watertight test's division); a reflection */
/* adds ERR_REFL ulps to the direction (the normal from float vertices,     */
/* cos theta0, the mirror formula, the normalisation); a refraction scales  */
/* the incoming direction error by the derivative of Snell's law            */
/* eta cos theta0 / cos theta2 and adds a third of the bound (6 eta^2 + 5)  */
/* 2^-24 / (2 cos theta2) of the rounding of sin^2 theta2, the normal's     */
/* ERR_NRM ulps turned by (A - 1) (A the same derivative), plus ERR_REFR    */
/* ulps.  A hit or near miss within FLAG_SIGMAS standard deviations of a    */
/* triangle edge is a decision float32 can take the other way and flags the */
/* ray.  For the hit distances the parity tests take the same estimate with */
/* one more term: a hit point's error across the ray moves it within the    */
/* hit plane by that error over cos theta0, and the children start there.   */
/* ------------------------------------------------------------------------ */
#define ULP32 0x1p-24
#define ERR_DIR0 2.0     /* ulps of the generated direction */
#define ERR_REFL 2.0     /* ulps a reflection adds */
#define ERR_REFR 1.0     /* ulps a refraction adds besides the Snell term */
#define ERR_NRM 1.5      /* ulps of a triangle normal computed from float vertices */
#define ERR_T 1.0        /* ulps of t from the watertight test's division */
#define FLAG_SIGMAS 4.0  /* standard deviations of a hit point that flag an edge */

/* one float32 ulp of x (the spacing of floats around |x|, at least 2^-149) */
static double ulp32(double x) {
  x = fabs(x);
  if (!(x >= 0x1p-126)) return 0x1p-149;
  int e;
  frexp(x, &e); /* x = f 2^e, 0.5 <= f < 1: floats in [2^(e-1), 2^e) are 2^(e-24) apart */
  return ldexp(1.0, e - 24);
}

/* standard deviation of the float32 point at distance t along (o, d) */
static double point_err(double e_org, double e_dir, double t, const double o[3], const double d[3]) {
  double m = 0.0;
  for (int i = 0; i < 3; ++i) m = fmax(m, fabs(o[i] + t * d[i]));
  const double r = 0.5 * ulp32(m), u = ERR_T * ulp32(t);
  return sqrt(e_org * e_org + t * t * e_dir * e_dir + r * r + u * u);
}

typedef struct {
  uint32_t tri;
  double t, margin;
  uint32_t flags;
} hit_t;

/* running state of a closest-hit query: the best hit so far, the second
   closest valid hit, the nearest near-edge candidate, a hit next to t_min */
typedef struct {
  hit_t h;
  double t2, t_edge;
  int near_tmin;
  double e_org, e_dir; /* the ray's float32 error estimate */
} hit_acc;

/* Is the plane point of triangle (v0, v1, v2) with barycentrics (b0, b1, b2)
   within barycentric margin FLAG_BARY of an edge, or closer to an edge than
   `err` metres (inside or outside; capped at FLAG_EMAX)?  The signed
   distance to the edge opposite vertex i is b_i times the altitude over
   that edge. */
static int near_edge(const double v0[3], const double v1[3], const double v2[3], double b0, double b1, double b2,
                     double m, double err) {
  if (m > -FLAG_BARY && m < FLAG_BARY) return 1;
  if (!(m > -0.5 && m < 0.5)) return 0;
  double e1[3], e2[3], e3[3], c[3];
  sub3(v1, v0, e1);
  sub3(v2, v0, e2);
  sub3(v2, v1, e3);
  cross3(e1, e2, c);
  const double twice_area = norm3(c);
  err = fmin(err, FLAG_EMAX);
  const double s0 = b0 * twice_area / norm3(e3), s1 = b1 * twice_area / norm3(e2), s2 = b2 * twice_area / norm3(e1);
  double smin = s0 < s1 ? s0 : s1;
  if (s2 < smin) smin = s2;
  return smin > -err && smin < err;
}

static void hit_begin(hit_acc* a) {
  a->h.tri = ORC_NONE;
  a->h.t = INFINITY;
  a->h.margin = 0.0;
  a->h.flags = 0u;
  a->t2 = INFINITY;
  a->t_edge = INFINITY;
  a->near_tmin = 0;
  a->e_org = 0.0;
  a->e_dir = 0.0;
}

/* one triangle of a closest-hit query (t > t_min; ties on t go to the
   smaller triangle id) */
static void hit_consider(const scene_t* s, uint32_t j, const double o[3], const double d[3], double t_min,
                         hit_acc* a) {
  double v0[3], v1[3], v2[3], t, b1, b2;
  tri_vertices(s, j, v0, v1, v2);
  if (!orc_tri_plane(o, d, v0, v1, v2, &t, &b1, &b2)) return;
  double b0 = 1.0 - b1 - b2;
  double m = b0 < b1 ? b0 : b1;
  if (b2 < m) m = b2;
  if (t > t_min - FLAG_TABS && t < a->t_edge &&
      near_edge(v0, v1, v2, b0, b1, b2, m, FLAG_SIGMAS * point_err(a->e_org, a->e_dir, t, o, d)))
    a->t_edge = t;
  if (m >= 0.0 && fabs(t - t_min) < FLAG_TABS) a->near_tmin = 1;
  if (m < 0.0 || !(t > t_min)) return;
  if (t < a->h.t || (t == a->h.t && j < a->h.tri)) {
    if (a->h.tri != ORC_NONE) a->t2 = a->h.t;
    a->h.t = t;
    a->h.tri = j;
    a->h.margin = m;
  } else if (t < a->t2) {
    a->t2 = t;
  }
}

/* parity flags of the finished query: a near-edge candidate that could be
   the closest, a near tie with the second closest triangle, a hit next to
   t_min */
static hit_t hit_finish(const hit_acc* a) {
  hit_t h = a->h;
  if (a->t_edge < INFINITY && a->t_edge <= h.t * (1.0 + FLAG_TREL)) h.flags |= SEG_EDGE;
  if (a->near_tmin) h.flags |= SEG_TMIN;
  if (h.tri != ORC_NONE && a->t2 - h.t <= FLAG_TREL * h.t) h.flags |= SEG_TIE;
  return h;
}

static hit_t closest_hit_bvh(const scene_t* s, const double o[3], const double d[3], double t_min, uint32_t skip,
                             double e_org, double e_dir);
static int occluded_bvh(const scene_t* s, const double p[3], const double dir[3], double t_min, double dist,
                        uint32_t skip, int* flag, double e_org, double e_dir);

/* Closest hit by brute force over all triangles: t > t_min, triangle != skip,
   ties on t go to the smaller triangle id.  Flags near-edge candidates (hit or
   miss within FLAG_BARY of an edge) that could be the closest, a near tie with
   the second closest triangle, and hits next to t_min. */
static hit_t closest_hit(const scene_t* s, const double o[3], const double d[3], double t_min, uint32_t skip,
                         double e_org, double e_dir) {
  if (s->bvh) return closest_hit_bvh(s, o, d, t_min, skip, e_org, e_dir);
  hit_acc a;
  hit_begin(&a);
  a.e_org = e_org;
  a.e_dir = e_dir;
  for (uint32_t j = 0; j < s->nt; ++j) {
    if (j == skip) continue;
    hit_consider(s, j, o, d, t_min, &a);
  }
  return hit_finish(&a);
}

/* exported for the tests: closest hit of one ray by brute force */
int orc_closest(const float* vertices, uint32_t n_vertices, const uint32_t* triangles, uint32_t n_triangles,
                const double o[3], const double d[3], double t_min, uint32_t skip, uint32_t* tri, double* t,
                uint32_t* flags) {
  scene_t s = {vertices, triangles, NULL, NULL, n_vertices, n_triangles, 0, NULL, 0};
  hit_t h = closest_hit(&s, o, d, t_min, skip, 0.0, 0.0);
  *tri = h.tri;
  *t = h.t;
  *flags = h.flags;
  return h.tri != ORC_NONE;
}

/* Standard deviation of the float32 point at distance t along the
   visibility segment from a hit point (error e_org) to the sensor (a float:
   no error) at distance dist: the segment is fixed by its two end points,
   so the error shrinks linearly toward the sensor. */
static double seg_err(double e_org, double t, double dist, const double p[3], const double dir[3]) {
  double m = 0.0;
  for (int i = 0; i < 3; ++i) m = fmax(m, fabs(p[i] + t * dir[i]));
  const double e = e_org * fmax(1.0 - t / dist, 0.0), r = 0.5 * ulp32(m), u = ERR_T * ulp32(t);
  return sqrt(e * e + r * r + u * u);
}

/* one triangle of an any-hit query on the open segment (t_min, dist) */
static void occ_consider(const scene_t* s, uint32_t j, const double p[3], const double dir[3], double t_min,
                         double dist, int* occ, int* flag, double e_org, double e_dir) {
  (void)e_dir;
  double v0[3], v1[3], v2[3], t, b1, b2;
  tri_vertices(s, j, v0, v1, v2);
  if (!orc_tri_plane(p, dir, v0, v1, v2, &t, &b1, &b2)) return;
  double b0 = 1.0 - b1 - b2;
  double m = b0 < b1 ? b0 : b1;
  if (b2 < m) m = b2;
  int inside_t = t > t_min && t < dist;
  int near_t = fabs(t - t_min) < FLAG_TABS || fabs(t - dist) < FLAG_TREL * dist;
  if ((inside_t || near_t) &&
      near_edge(v0, v1, v2, b0, b1, b2, m, FLAG_SIGMAS * seg_err(e_org, t, dist, p, dir)))
    *flag = 1;
  if (m >= 0.0 && near_t) *flag = 1;
  if (m >= 0.0 && inside_t) *occ = 1;
}

/* Any hit on the open segment from p (on triangle skip) to the sensor at
   distance dist.  Sets *flag when a triangle lies within the flag margins. */
static int occluded(const scene_t* s, const double p[3], const double dir[3], double t_min, double dist, uint32_t skip,
                    int* flag, double e_org, double e_dir) {
  if (s->bvh) return occluded_bvh(s, p, dir, t_min, dist, skip, flag, e_org, e_dir);
  int occ = 0;
  for (uint32_t j = 0; j < s->nt; ++j) {
    if (j == skip) continue;
    occ_consider(s, j, p, dir, t_min, dist, &occ, flag, e_org, e_dir);
  }
  return occ;
}

/* ------------------------------------------------------------------------ */
/* CPU BVH: the timed CPU baseline traces with the oracle's physics through  */
/* a bounding volume hierarchy instead of the brute-force loops above.       */
/* Binary tree, binned SAH (16 bins per axis over the centroids), leaves of  */
/* at most 4 triangles, float boxes rounded outward.  Every triangle's box    */
/* is grown by 1e-4 of its largest extent plus 2 FLAG_EMAX, which holds every */
/* point of its plane within barycentric margin FLAG_BARY, or within the      */
/* largest edge distance FLAG_EMAX that flags, of the triangle (built for    */
/* the flags; the fast mode's tree grows them by 1e-6 m only):               */
/* so a query that keeps visiting boxes up to (1 + 1e-5) times the best t     */
/* sees every triangle the brute-force loops would count (the closest hit,   */
/* the second closest, near-edge candidates, hits next to t_min) and gives   */
/* the same hit and the same flags.  In the fast mode (timing) the pruning   */
/* is strict, any-hit queries stop at the first occluder and the flags are   */
/* not meaningful; the hits are the same.                                    */
/* ------------------------------------------------------------------------ */
#define BVH_BINS 16
#define BVH_LEAF 4
#define BVH_STACK 128
#define WTAB_CELLS 8192

typedef struct {
  float lo[3], hi[3];
  uint32_t first; /* leaf: first index into idx; internal: left child (right = first + 1) */
  uint32_t count; /* leaf: number of triangles (> 0); internal: 0 */
} bnode_t;

struct orc_bvh {
  bnode_t* nodes;
  uint32_t* idx;
  uint32_t n_nodes, depth;
  int exact; /* boxes grown for the parity flags */
  /* tabulated lobe integrals for the fast mode: per material the integral of
     the density from 0 to x_k = k (pi/2) / WTAB_CELLS and the density there */
  double* wtab;
  uint32_t nm;
};

typedef struct {
  double lo[3], hi[3];
} box_t;

static void box_empty(box_t* b) {
  for (int i = 0; i < 3; ++i) {
    b->lo[i] = INFINITY;
    b->hi[i] = -INFINITY;
  }
}

static void box_grow(box_t* b, const box_t* c) {
  for (int i = 0; i < 3; ++i) {
    if (c->lo[i] < b->lo[i]) b->lo[i] = c->lo[i];
    if (c->hi[i] > b->hi[i]) b->hi[i] = c->hi[i];
  }
}

static double box_area(const box_t* b) {
  double e0 = b->hi[0] - b->lo[0], e1 = b->hi[1] - b->lo[1], e2 = b->hi[2] - b->lo[2];
  if (!(e0 >= 0.0)) return 0.0;
  return 2.0 * (e0 * e1 + e1 * e2 + e2 * e0);
}

typedef struct {
  box_t* tbox; /* grown triangle boxes */
  double* cen; /* [T][3] centroids of the grown boxes */
  uint32_t* idx;
  bnode_t* nodes;
  uint32_t n_nodes, cap, depth;
} build_t;

/* two consecutive node slots (left and right child) */
static uint32_t node_alloc2(build_t* B) {
  uint32_t i;
#ifdef _OPENMP
#pragma omp atomic capture
#endif
  {
    i = B->n_nodes;
    B->n_nodes += 2;
  }
  return i;
}

static void set_node_box(bnode_t* n, const box_t* b) {
  for (int i = 0; i < 3; ++i) {
    n->lo[i] = nextafterf((float)b->lo[i], -INFINITY);
    n->hi[i] = nextafterf((float)b->hi[i], INFINITY);
  }
}

/* builds the subtree of idx[first, first + count) into node ni */
static void build_node(build_t* B, uint32_t ni, uint32_t first, uint32_t count, uint32_t depth) {
  box_t bb, cb;
  box_empty(&bb);
  box_empty(&cb);
  for (uint32_t i = first; i < first + count; ++i) {
    const uint32_t j = B->idx[i];
    box_grow(&bb, &B->tbox[j]);
    box_t c = {{B->cen[3 * j], B->cen[3 * j + 1], B->cen[3 * j + 2]}, {B->cen[3 * j], B->cen[3 * j + 1], B->cen[3 * j + 2]}};
    box_grow(&cb, &c);
  }
  bnode_t* n = &B->nodes[ni];
  set_node_box(n, &bb);
  if (depth > B->depth) B->depth = depth;
  if (count <= BVH_LEAF) {
    n->first = first;
    n->count = count;
    return;
  }
  /* binned SAH over the centroid bounds */
  int best_axis = -1, best_split = 0;
  double best_cost = INFINITY;
  for (int ax = 0; ax < 3; ++ax) {
    double ext = cb.hi[ax] - cb.lo[ax];
    if (!(ext > 0.0)) continue;
    box_t bin_box[BVH_BINS];
    uint32_t bin_n[BVH_BINS] = {0};
    for (int k = 0; k < BVH_BINS; ++k) box_empty(&bin_box[k]);
    const double scale = BVH_BINS / ext;
    for (uint32_t i = first; i < first + count; ++i) {
      const uint32_t j = B->idx[i];
      int k = (int)((B->cen[3 * j + ax] - cb.lo[ax]) * scale);
      if (k >= BVH_BINS) k = BVH_BINS - 1;
      if (k < 0) k = 0;
      bin_n[k]++;
      box_grow(&bin_box[k], &B->tbox[j]);
    }
    double right_area[BVH_BINS];
    uint32_t right_n[BVH_BINS];
    box_t acc;
    box_empty(&acc);
    uint32_t cnt = 0;
    for (int k = BVH_BINS - 1; k > 0; --k) {
      box_grow(&acc, &bin_box[k]);
      cnt += bin_n[k];
      right_area[k] = box_area(&acc);
      right_n[k] = cnt;
    }
    box_empty(&acc);
    cnt = 0;
    for (int k = 0; k < BVH_BINS - 1; ++k) {
      box_grow(&acc, &bin_box[k]);
      cnt += bin_n[k];
      if (cnt == 0 || right_n[k + 1] == 0) continue;
      double cost = box_area(&acc) * cnt + right_area[k + 1] * right_n[k + 1];
      if (cost < best_cost) {
        best_cost = cost;
        best_axis = ax;
        best_split = k + 1;
      }
    }
  }
  uint32_t mid;
  if (best_axis < 0) {
    mid = first + count / 2; /* all centroids equal: split the list */
  } else {
    const double scale = BVH_BINS / (cb.hi[best_axis] - cb.lo[best_axis]);
    uint32_t i = first, e = first + count;
    while (i < e) {
      const uint32_t j = B->idx[i];
      int k = (int)((B->cen[3 * j + best_axis] - cb.lo[best_axis]) * scale);
      if (k >= BVH_BINS) k = BVH_BINS - 1;
      if (k < best_split) {
        ++i;
      } else {
        B->idx[i] = B->idx[--e];
        B->idx[e] = j;
      }
    }
    mid = i;
    if (mid == first || mid == first + count) mid = first + count / 2;
  }
  const uint32_t left = node_alloc2(B);
  n->first = left;
  n->count = 0;
  const uint32_t nl = mid - first, nr = first + count - mid;
#ifdef _OPENMP
  if (count > 65536) {
#pragma omp task
    build_node(B, left, first, nl, depth + 1);
#pragma omp task
    build_node(B, left + 1, mid, nr, depth + 1);
#pragma omp taskwait
    return;
  }
#endif
  build_node(B, left, first, nl, depth + 1);
  build_node(B, left + 1, mid, nr, depth + 1);
}

/* Builds the BVH of a triangle soup (and, for the fast mode, the window
   tables of the materials).  Returns NULL on bad input. */
orc_bvh* orc_bvh_build(const float* vertices, uint32_t n_vertices, const uint32_t* triangles, uint32_t n_triangles,
                       const orc_material* materials, uint32_t n_materials, uint32_t* depth_out, int exact) {
  if (n_triangles == 0) return NULL;
  for (size_t i = 0; i < 3 * (size_t)n_triangles; ++i)
    if (triangles[i] >= n_vertices) return NULL;
  build_t B;
  memset(&B, 0, sizeof B);
  B.tbox = (box_t*)malloc(sizeof(box_t) * n_triangles);
  B.cen = (double*)malloc(sizeof(double) * 3 * n_triangles);
  B.idx = (uint32_t*)malloc(sizeof(uint32_t) * n_triangles);
  B.cap = 2 * n_triangles;
  B.nodes = (bnode_t*)calloc(B.cap, sizeof(bnode_t));
  scene_t s = {vertices, triangles, NULL, NULL, n_vertices, n_triangles, 0, NULL, 0};
  for (uint32_t j = 0; j < n_triangles; ++j) {
    double v0[3], v1[3], v2[3];
    tri_vertices(&s, j, v0, v1, v2);
    box_t b;
    double ext = 0.0;
    for (int i = 0; i < 3; ++i) {
      b.lo[i] = fmin(v0[i], fmin(v1[i], v2[i]));
      b.hi[i] = fmax(v0[i], fmax(v1[i], v2[i]));
      ext = fmax(ext, b.hi[i] - b.lo[i]);
    }
    const double grow = exact ? 1e-4 * ext + 2.0 * FLAG_EMAX : 1e-6;
    for (int i = 0; i < 3; ++i) {
      b.lo[i] -= grow;
      b.hi[i] += grow;
      B.cen[3 * (size_t)j + i] = 0.5 * (b.lo[i] + b.hi[i]);
    }
    B.tbox[j] = b;
    B.idx[j] = j;
  }
  B.n_nodes = 1;
#ifdef _OPENMP
#pragma omp parallel
#pragma omp single
#endif
  build_node(&B, 0, 0, n_triangles, 1);
  free(B.tbox);
  free(B.cen);
  orc_bvh* h = (orc_bvh*)calloc(1, sizeof(orc_bvh));
  h->nodes = B.nodes;
  h->idx = B.idx;
  h->n_nodes = B.n_nodes;
  h->depth = B.depth;
  h->exact = exact;
  if (depth_out) *depth_out = B.depth;
  if (B.depth + 1 >= BVH_STACK) {
    free(h->nodes);
    free(h->idx);
    free(h);
    return NULL;
  }
  /* window tables: G_k = integral of the density over [0, x_k], summed cell by
     cell with the oracle's own window integral, and the density f_k */
  h->nm = n_materials;
  if (materials && n_materials) {
    const double hx = 0.5 * M_PI / WTAB_CELLS;
    h->wtab = (double*)malloc(sizeof(double) * 2 * (WTAB_CELLS + 1) * n_materials);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int mi = 0; mi < (int)n_materials; ++mi) {
      double* G = h->wtab + (size_t)mi * 2 * (WTAB_CELLS + 1);
      double* F = G + (WTAB_CELLS + 1);
      G[0] = 0.0;
      for (int k = 0; k <= WTAB_CELLS; ++k) {
        F[k] = orc_brdf_density(&materials[mi], k * hx);
        if (k < WTAB_CELLS) G[k + 1] = G[k] + orc_brdf_window(&materials[mi], (k + 0.5) * hx, hx);
      }
    }
  }
  return h;
}

void orc_bvh_free(orc_bvh* h) {
  if (!h) return;
  free(h->nodes);
  free(h->idx);
  free(h->wtab);
  free(h);
}

/* integral of material mi's density over [0, x], 0 <= x <= pi/2: cubic
   Hermite interpolation of the tabulated integral (its derivative is the
   density) */
static double wtab_prim(const orc_bvh* h, uint32_t mi, double x) {
  const double hx = 0.5 * M_PI / WTAB_CELLS;
  const double* G = h->wtab + (size_t)mi * 2 * (WTAB_CELLS + 1);
  const double* F = G + (WTAB_CELLS + 1);
  double u = x / hx;
  if (!(u > 0.0)) return 0.0;
  if (u >= WTAB_CELLS) return G[WTAB_CELLS];
  int k = (int)u;
  double t = u - k, t2 = t * t, t3 = t2 * t;
  return (2 * t3 - 3 * t2 + 1) * G[k] + (t3 - 2 * t2 + t) * hx * F[k] + (-2 * t3 + 3 * t2) * G[k + 1] +
         (t3 - t2) * hx * F[k + 1];
}

/* W(w) of Eq. 4: the oracle's quadrature, or in the fast mode the table */
static double window(const scene_t* s, uint32_t mi, double w, double b) {
  const orc_material* m = &s->mat[mi];
  if (!(s->fast && s->bvh && s->bvh->wtab)) return orc_brdf_window(m, w, b);
  double lo = w - 0.5 * b, hi = w + 0.5 * b;
  if (lo < -M_PI / 2) lo = -M_PI / 2;
  if (hi > M_PI / 2) hi = M_PI / 2;
  if (!(hi > lo)) return 0.0;
  double gh = hi >= 0.0 ? wtab_prim(s->bvh, mi, hi) : -wtab_prim(s->bvh, mi, -hi);
  double gl = lo >= 0.0 ? wtab_prim(s->bvh, mi, lo) : -wtab_prim(s->bvh, mi, -lo);
  return gh - gl;
}

/* entry and exit distance of the ray through a node box; 0 if it misses
   [t_lo, t_hi] */
static int node_range(const bnode_t* n, const double o[3], const double inv[3], double t_lo, double t_hi,
                      double* t_in) {
  double a = t_lo, b = t_hi;
  for (int i = 0; i < 3; ++i) {
    double x0, x1;
    if (isinf(inv[i])) {
      if (o[i] < (double)n->lo[i] || o[i] > (double)n->hi[i]) return 0;
      continue;
    }
    x0 = ((double)n->lo[i] - o[i]) * inv[i];
    x1 = ((double)n->hi[i] - o[i]) * inv[i];
    if (x0 > x1) {
      double t = x0;
      x0 = x1;
      x1 = t;
    }
    if (x0 > a) a = x0;
    if (x1 < b) b = x1;
    if (a > b) return 0;
  }
  *t_in = a;
  return 1;
}

static void inv_dir(const double d[3], double inv[3]) {
  for (int i = 0; i < 3; ++i) inv[i] = d[i] != 0.0 ? 1.0 / d[i] : INFINITY;
}

static hit_t closest_hit_bvh(const scene_t* s, const double o[3], const double d[3], double t_min, uint32_t skip,
                             double e_org, double e_dir) {
  const orc_bvh* B = s->bvh;
  hit_acc a;
  hit_begin(&a);
  a.e_org = e_org;
  a.e_dir = e_dir;
  double inv[3];
  inv_dir(d, inv);
  const double t_lo = s->fast ? t_min : t_min - 1e-5;
  uint32_t stack[BVH_STACK];
  double stack_t[BVH_STACK];
  int sp = 0;
  double t0;
  if (!node_range(&B->nodes[0], o, inv, t_lo, INFINITY, &t0)) return hit_finish(&a);
  stack[sp] = 0;
  stack_t[sp++] = t0;
  while (sp > 0) {
    --sp;
    const double limit = s->fast ? a.h.t : fmax(a.h.t * (1.0 + 1e-5), t_min + 1e-5) + 1e-9;
    if (stack_t[sp] > limit) continue;
    const bnode_t* n = &B->nodes[stack[sp]];
    if (n->count) {
      for (uint32_t i = n->first; i < n->first + n->count; ++i) {
        const uint32_t j = B->idx[i];
        if (j != skip) hit_consider(s, j, o, d, t_min, &a);
      }
      continue;
    }
    double tl, tr;
    const int hl = node_range(&B->nodes[n->first], o, inv, t_lo, limit, &tl);
    const int hr = node_range(&B->nodes[n->first + 1], o, inv, t_lo, limit, &tr);
    if (hl && hr) {
      const int near_left = tl <= tr;
      stack[sp] = near_left ? n->first + 1 : n->first;
      stack_t[sp++] = near_left ? tr : tl;
      stack[sp] = near_left ? n->first : n->first + 1;
      stack_t[sp++] = near_left ? tl : tr;
    } else if (hl) {
      stack[sp] = n->first;
      stack_t[sp++] = tl;
    } else if (hr) {
      stack[sp] = n->first + 1;
      stack_t[sp++] = tr;
    }
  }
  return hit_finish(&a);
}

static int occluded_bvh(const scene_t* s, const double p[3], const double dir[3], double t_min, double dist,
                        uint32_t skip, int* flag, double e_org, double e_dir) {
  const orc_bvh* B = s->bvh;
  double inv[3];
  inv_dir(dir, inv);
  const double t_lo = s->fast ? t_min : t_min - 1e-5;
  const double t_hi = s->fast ? dist : dist * (1.0 + 1e-5) + 1e-5;
  uint32_t stack[BVH_STACK];
  int sp = 0, occ = 0;
  double t0;
  if (!node_range(&B->nodes[0], p, inv, t_lo, t_hi, &t0)) return 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const bnode_t* n = &B->nodes[stack[--sp]];
    if (n->count) {
      for (uint32_t i = n->first; i < n->first + n->count; ++i) {
        const uint32_t j = B->idx[i];
        if (j != skip) occ_consider(s, j, p, dir, t_min, dist, &occ, flag, e_org, e_dir);
      }
      if (occ && s->fast) return 1;
      continue;
    }
    for (uint32_t c = n->first; c < n->first + 2; ++c)
      if (node_range(&B->nodes[c], p, inv, t_lo, t_hi, &t0)) stack[sp++] = c;
  }
  return occ;
}

/* ------------------------------------------------------------------------ */
/* per-column work                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  double o[3], d[3], E, L;
  int32_t medium;
  uint32_t prev, path, bounce;
  double e_org, e_dir; /* float32 error estimate (see above) */
  double e_tol;        /* the origin's error for the distance tolerances (moved within hit planes) */
} oray_t;

typedef struct {
  uint32_t k;
  double range, E;
} oret_t;

typedef struct {
  oret_t* ret;
  size_t n_ret, cap_ret;
  orc_segment* seg;
  size_t n_seg, cap_seg;
  uint8_t* flagged;   /* [Ns] */
  double* tally;      /* [Ns][4]: returned, absorbed, escaped, terminated */
  uint64_t queries, shadow_queries;
  int keep_segs;      /* store the segments (else only count them) */
} column_t;

static void push_ret(column_t* c, uint32_t k, double range, double E) {
  if (c->n_ret == c->cap_ret) {
    c->cap_ret = c->cap_ret ? 2 * c->cap_ret : 256;
    c->ret = (oret_t*)realloc(c->ret, c->cap_ret * sizeof(oret_t));
  }
  c->ret[c->n_ret].k = k;
  c->ret[c->n_ret].range = range;
  c->ret[c->n_ret].E = E;
  c->n_ret++;
}

static void push_seg(column_t* c, const orc_segment* s) {
  if (!c->keep_segs) {
    c->n_seg++;
    return;
  }
  if (c->n_seg == c->cap_seg) {
    c->cap_seg = c->cap_seg ? 2 * c->cap_seg : 256;
    c->seg = (orc_segment*)realloc(c->seg, c->cap_seg * sizeof(orc_segment));
  }
  c->seg[c->n_seg++] = *s;
}

static double refr_index(const scene_t* s, int32_t medium) {
  return medium == ORC_AIR ? 1.0 : sqrt(s->mat[medium].eps_r);
}

/* field attenuation constant alpha = pi sqrt(eps_r) tan(delta) / lambda, lambda = c / f */
static double alpha_np(const scene_t* s, int32_t medium, double freq) {
  if (medium == ORC_AIR) return 0.0;
  const double c0 = 299792458.0;
  const orc_material* m = &s->mat[medium];
  return M_PI * sqrt(m->eps_r) * m->loss_tangent * freq / c0;
}

/* Gaussian receive weight of beam a for a return arriving from pt: the
   transmit density of the D3 cone read as the receive pattern.  delta is the
   angle between pt - sensor and the beam axis; for an elliptic beam (aspect
   a != 1) the spread along the offset's direction psi around the axis
   (psi = 0 along increasing azimuth, pi/2 along increasing elevation) is
   sigma / sqrt(cos^2 psi + sin^2 psi / a^2). */
static double receive_weight(const orc_params* p, const orc_pose* pose, uint32_t a, const double axis[3],
                             const double sensor[3], const double pt[3]) {
  double sigma = orc_d3_sigma(p->beam_width, p->beam_prob);
  if (sigma == 0.0) return 0.0;
  double v[3];
  sub3(pt, sensor, v);
  double delta = orc_angle(v, axis);
  double f = 1.0;
  if (p->beam_aspect != 1.0) {
    double phi = 2.0 * M_PI * (double)a / (double)p->n_azimuth, th = p->elevation;
    double ea_s[3] = {-sin(phi), cos(phi), 0.0};
    double ee_s[3] = {-sin(th) * cos(phi), -sin(th) * sin(phi), cos(th)};
    double ea[3], ee[3];
    quat_rotate(pose->q, ea_s, ea);
    quat_rotate(pose->q, ee_s, ee);
    double ca = dot3(v, ea), ce = dot3(v, ee);
    double perp2 = ca * ca + ce * ce;
    if (perp2 > 0.0) f = (ca * ca + ce * ce / (p->beam_aspect * p->beam_aspect)) / perp2;
  }
  return exp(-0.5 * delta * delta * f / (sigma * sigma));
}

/* the receive weight of beam a of the pose for a return from pt (exported for the pins) */
double orc_receive_weight(const orc_params* p, const orc_pose* pose, uint32_t a, const double pt[3]) {
  double axis[3];
  orc_beam_axis(p, pose, a, axis);
  return receive_weight(p, pose, a, axis, pose->p, pt);
}

/* Speckle (Sec. III-C noise model): the energy of one return is multiplied
   by an Exp(1) factor -ln u (fully developed speckle: exponential intensity
   with mean one, so the expected image is unchanged).  u is word `which` of
   the Philox block of counter (scan_id, a, k, 1 | (path << 8 | bounce) << 8):
   one block per segment, word 0 for its traveled-path return, word 1 for its
   air-path return. */
double orc_speckle_factor(const orc_params* p, uint32_t a, uint32_t k, uint32_t path, uint32_t bounce, int which) {
  uint32_t x[4];
  draw(p, a, k, 1u | (((path << 8) | bounce) << 8), x);
  return -log(orc_u24(x[which]));
}

/* Optional range weight of a return at range r (metres): Eq. 1's power
   falloff R^-k made explicit, normalised at 1 m and never above one:
   (1 / r)^k for r > 1 m, 1 otherwise.  k = 0 (the default) leaves the image
   to the ray density alone, as Sec. III-A describes. */
double orc_range_weight(const orc_params* p, double r) {
  if (p->range_falloff == 0.0 || !(r > 1.0)) return 1.0;
  return pow(r, -p->range_falloff);
}

/* Sec. III-A: trace the ray tree of every initial ray of azimuth a. */
static void trace_column(const scene_t* s, const orc_params* p, const orc_pose* pose, uint32_t a, column_t* col) {
  const double r_max = (double)p->n_bins * p->bin_size;
  const double r_lim = ((p->flags & ORC_MULTIPATH) ? 2.0 : 1.0) * r_max;
  const double b = p->beam_width;
  double axis[3];
  orc_beam_axis(p, pose, a, axis);
  const double* sensor = pose->p;

  size_t cap = 64;
  oray_t* stack = (oray_t*)malloc(cap * sizeof(oray_t));

  const uint32_t stride = p->ray_stride > 1 ? p->ray_stride : 1u;
  for (uint32_t k = 0; k < p->rays_per_beam; k += stride) {
    double* tal = col->tally + 4 * (size_t)k;
    int flagged = 0;
    size_t sp = 0;
    oray_t root;
    orc_d3_ray(p, pose, a, k, root.o, root.d, NULL, NULL);
    root.E = 1.0 / (double)p->rays_per_beam; /* Sec. III-A: ray energies sum to E0 = 1 */
    root.L = 0.0;
    root.medium = ORC_AIR;
    root.prev = ORC_NONE;
    root.path = 0;
    root.bounce = 0;
    root.e_org = 0.0;
    root.e_tol = 0.0;
    root.e_dir = ERR_DIR0 * ULP32;
    stack[sp++] = root;

    while (sp > 0) {
      oray_t ray = stack[--sp];
      orc_segment seg = {a, k, ray.path, ray.bounce, ORC_NONE, 0u, INFINITY, ray.E, 0.0, 0.0, 0.0,
                         ray.e_tol, ray.e_dir, 2.0 * alpha_np(s, ray.medium, p->freq_hz)};
      double n_cur = refr_index(s, ray.medium);
      double t_lim = (r_lim - ray.L) / n_cur; /* past it no return can reach the image */
      hit_t h = closest_hit(s, ray.o, ray.d, p->t_min, ray.prev, ray.e_org, ray.e_dir);
      col->queries++;
      seg.flags = h.flags;
      if (h.tri != ORC_NONE && fabs(h.t - t_lim) <= FLAG_TREL * t_lim) seg.flags |= SEG_TLIM;
      if (h.tri == ORC_NONE || h.t >= t_lim) {
        tal[2] += ray.E; /* escaped */
        push_seg(col, &seg);
        if (seg.flags & ~SEG_TALLY) flagged |= 1;
        if (seg.flags & SEG_TALLY) flagged |= 2;
        continue;
      }
      seg.tri = h.tri;
      seg.t = h.t;
      const double e_hit = point_err(ray.e_org, ray.e_dir, h.t, ray.o, ray.d);
      if (FLAG_SIGMAS * e_hit > FLAG_EMAX) seg.flags |= SEG_ERR;
      /* for the distance tolerances: the error of the hit point within the
         hit plane, where the children start -- a ray meeting the plane at
         cos theta0 moves its hit point along the plane by its error across
         the ray over cos theta0 */
      double e_tol_hit;
      {
        double nh[3];
        tri_normal(s, h.tri, nh);
        e_tol_hit = point_err(ray.e_tol, ray.e_dir, h.t, ray.o, ray.d) / fmax(fabs(dot3(ray.d, nh)), 1e-6);
      }

      double pt[3];
      for (int i = 0; i < 3; ++i) pt[i] = ray.o[i] + h.t * ray.d[i];
      double L1 = ray.L + n_cur * h.t;
      /* attenuation inside a lossy medium: E <- E exp(-2 alpha d) */
      double E1 = ray.E;
      if (ray.medium != ORC_AIR) {
        E1 = ray.E * exp(-2.0 * alpha_np(s, ray.medium, p->freq_hz) * h.t);
        tal[1] += ray.E - E1;
      }

      const uint32_t mid = s->mat_id[h.tri];
      const orc_material* m = &s->mat[mid];
      double n[3];
      tri_normal(s, h.tri, n);
      double cos_i = -dot3(ray.d, n);
      if (fabs(cos_i) < FLAG_COS) seg.flags |= SEG_GRAZE;
      /* a segment inside a medium: its length may move by FLAG_SIGMAS
         standard deviations of its float32 hit point over |cos theta0|, and
         the energy the medium absorbs over it (and every energy after it) by
         2 alpha E_end as much; flagged for the per-ray tallies when that can
         reach half their tolerance */
      if (ray.medium != ORC_AIR) {
        double dt = FLAG_SIGMAS * e_hit / fmax(fabs(cos_i), 1e-12);
        if (2.0 * alpha_np(s, ray.medium, p->freq_hz) * E1 * dt > FLAG_TALLY / (double)p->rays_per_beam)
          seg.flags |= SEG_TALLY;
      }
      int entering = cos_i > 0.0;
      double n1 = n_cur, n2;
      int32_t next_medium;
      if (entering) {
        n2 = sqrt(m->eps_r);
        next_medium = (int32_t)mid;
      } else {
        for (int i = 0; i < 3; ++i) n[i] = -n[i];
        cos_i = -cos_i;
        n2 = 1.0;
        next_medium = ORC_AIR;
      }

      double R, cos_t = 0.0, sin2_t = 0.0, e_refr_dir = 0.0;
      int tir = 0;
      if (m->pec) {
        R = 1.0;
      } else {
        tir = orc_fresnel(n1, n2, cos_i, &R, &cos_t, &sin2_t);
        if (fabs(sin2_t - 1.0) < FLAG_TIR) seg.flags |= SEG_TIR;
        /* Snell's law is ill-conditioned next to the critical angle.  In
           float32, sin^2 theta2 = eta^2 (1 - cos^2 theta0) carries an error
           of at most (6 eta^2 + 5) 2^-24 (cos theta0 itself off by 3 ulps,
           twice amplified by eta^2, plus the roundings of the products), and
           theta2 moves by that over 2 cos theta2 sin theta2 ~ 2 cos theta2:
           the refracted child is flagged when this angle error exceeds the
           relative hit-distance tolerance (a direction off by d theta moves
           the next hit distance by about d theta of itself) */
        if (!tir && (p->flags & ORC_REFRACTION)) {
          double eta = n1 / n2;
          const double snell = (6.0 * eta * eta + 5.0) * ULP32 / (2.0 * cos_t);
          /* Snell's derivative scales the incoming direction's error; a normal
             turned by dn turns the refracted direction by (A - 1) dn */
          const double A = eta * cos_i / cos_t;
          const double amp = ray.e_dir * A, nrm = ERR_NRM * ULP32 * fabs(A - 1.0);
          e_refr_dir = sqrt(amp * amp + nrm * nrm + snell * snell / 9.0 + ERR_REFR * ERR_REFR * ULP32 * ULP32);
          if (!(snell <= FLAG_TDIR)) seg.flags |= SEG_SNELL;
        }
      }
      double T = (m->pec || tir) ? 0.0 : 1.0 - R;
      int can_refract = !m->pec && !tir;

      double d_refl[3], d_refr[3] = {0, 0, 0};
      orc_reflect(ray.d, n, d_refl);
      normalize3(d_refl);
      if (can_refract) {
        orc_refract(ray.d, n, n1 / n2, cos_i, cos_t, d_refr);
        normalize3(d_refr);
      }

      /* traveled-path return: omega = theta0 + theta1 = 2 theta0, range = L1 */
      double dn[3];
      for (int i = 0; i < 3; ++i) dn[i] = -n[i];
      double theta0 = orc_angle(ray.d, dn);
      double ret_t = E1 * R * window(s, mid, 2.0 * theta0, b);

      /* air-path return (multipath), bounce >= 1 only */
      double ret_a = 0.0, range_a = 0.0;
      int air_uses_T = 0;
      if ((p->flags & ORC_MULTIPATH) && ray.bounce >= 1) {
        int candidate = 0;
        const double* dir_out = NULL;
        double base = 0.0, cap_a = 0.0;
        double v[3];
        sub3(sensor, pt, v);
        double dist = norm3(v);
        double side = dot3(v, n) / dist;
        if (entering && ray.medium == ORC_AIR) {
          candidate = 1;
          dir_out = d_refl;
          base = E1 * R;
          cap_a = E1 * R - ret_t;
          if (fabs(side) < FLAG_COS) seg.flags |= SEG_VIS;
          if (side <= 0.0) candidate = 0;
        } else if (!entering && ray.medium != ORC_AIR && can_refract) {
          candidate = 1;
          air_uses_T = 1;
          dir_out = d_refr;
          base = E1 * T;
          cap_a = E1 * T;
          if (fabs(side) < FLAG_COS) seg.flags |= SEG_VIS;
          if (side >= 0.0) candidate = 0;
        }
        if (candidate) {
          double w_a = window(s, mid, orc_angle(dir_out, v), b);
          if (w_a > 0.0) {
            double dir[3] = {v[0] / dist, v[1] / dist, v[2] / dist};
            int vflag = 0;
            int occ = occluded(s, pt, dir, p->t_min, dist, h.tri, &vflag, e_hit, hypot(e_hit / dist, ULP32));
            col->shadow_queries++;
            if (vflag) seg.flags |= SEG_VIS;
            if (!occ) {
              double g = receive_weight(p, pose, a, axis, sensor, pt);
              ret_a = base * w_a * g;
              if (ret_a > cap_a) ret_a = cap_a;
              range_a = 0.5 * (L1 + dist);
            }
          }
        }
      }

      /* record the returns (Sec. III-A: collected in a list) */
      tal[0] += ret_t + ret_a;
      seg.cos_i = cos_i;
      seg.ret_t = ret_t;
      seg.ret_a = ret_a;
      if (ret_t > 0.0) {
        double e = ret_t;
        if (p->flags & ORC_SPECKLE) e *= orc_speckle_factor(p, a, k, ray.path, ray.bounce, 0);
        e *= orc_range_weight(p, L1);
        push_ret(col, k, L1, e);
      }
      if (ret_a > 0.0) {
        double e = ret_a;
        if (p->flags & ORC_SPECKLE) e *= orc_speckle_factor(p, a, k, ray.path, ray.bounce, 1);
        e *= orc_range_weight(p, range_a);
        push_ret(col, k, range_a, e);
      }

      /* children: the remaining energy goes on (Sec. III-A) */
      double e_refl = E1 * R - ret_t - (air_uses_T ? 0.0 : ret_a);
      double e_refr = E1 * T - (air_uses_T ? ret_a : 0.0);
      if (e_refl < 0.0) e_refl = 0.0;
      if (e_refr < 0.0) e_refr = 0.0;
      int deeper = ray.bounce + 1 < p->max_bounces;
      if (fabs(L1 - r_max) <= FLAG_TREL * r_max) seg.flags |= SEG_RMAX;
      int in_range = L1 < r_max;
      int spawn_refl = deeper && in_range && e_refl >= p->min_energy;
      int spawn_refr = deeper && in_range && can_refract && (p->flags & ORC_REFRACTION) && e_refr >= p->min_energy;
      if (p->min_energy > 0.0 && deeper && in_range) {
        if (fabs(e_refl - p->min_energy) < 1e-5 * p->min_energy) seg.flags |= SEG_EMIN;
        if (can_refract && fabs(e_refr - p->min_energy) < 1e-5 * p->min_energy) seg.flags |= SEG_EMIN;
      }
      if (!spawn_refl) tal[3] += e_refl;
      if (!spawn_refr) tal[3] += e_refr;

      push_seg(col, &seg);
      if (seg.flags & ~SEG_TALLY) flagged |= 1;   /* bit 0: paths, energies, images */
      if (seg.flags & SEG_TALLY) flagged |= 2;    /* bit 1: the tallies only */

      if (sp + 2 > cap) {
        cap *= 2;
        stack = (oray_t*)realloc(stack, cap * sizeof(oray_t));
      }
      if (spawn_refr) {
        oray_t c;
        memcpy(c.o, pt, sizeof pt);
        memcpy(c.d, d_refr, sizeof d_refr);
        c.E = e_refr;
        c.L = L1;
        c.medium = next_medium;
        c.prev = h.tri;
        c.path = (ray.path << 1) | 1u;
        c.bounce = ray.bounce + 1;
        c.e_org = e_hit;
        c.e_tol = e_tol_hit;
        c.e_dir = e_refr_dir;
        stack[sp++] = c;
      }
      if (spawn_refl) {
        oray_t c;
        memcpy(c.o, pt, sizeof pt);
        memcpy(c.d, d_refl, sizeof d_refl);
        c.E = e_refl;
        c.L = L1;
        c.medium = ray.medium;
        c.prev = h.tri;
        c.path = ray.path << 1;
        c.bounce = ray.bounce + 1;
        c.e_org = e_hit;
        c.e_tol = e_tol_hit;
        c.e_dir = sqrt(ray.e_dir * ray.e_dir + ERR_REFL * ERR_REFL * ULP32 * ULP32);
        stack[sp++] = c;
      }
    }
    col->flagged[k] = (uint8_t)flagged;
  }
  free(stack);
}

/* ------------------------------------------------------------------------ */
/* Sec. III-B: polar image by lookup and summation, starting at 0.          */
/* img sums every return; img_masked leaves out the returns of flagged      */
/* initial rays.  A return of an unflagged ray within a small window of a   */
/* bin edge also adds its energy to the slack of both neighbouring bins.    */
/* ------------------------------------------------------------------------ */
static void bin_column(const orc_params* p, const column_t* col, double* img, double* img_masked, double* slack) {
  for (size_t i = 0; i < col->n_ret; ++i) {
    const oret_t* r = &col->ret[i];
    const int flagged = col->flagged[r->k] & 1;
    double x = r->range / p->bin_size;
    double fb = floor(x);
    if (fb >= 0.0 && fb < (double)p->n_bins) {
      img[(size_t)fb] += r->E;
      if (!flagged && img_masked) img_masked[(size_t)fb] += r->E;
    }
    if (slack && !flagged) {
      double edge = floor(x + 0.5);
      double tol = 1e-4 > 4e-6 * x ? 1e-4 : 4e-6 * x;
      if (fabs(x - edge) < tol) {
        long lo = (long)edge - 1, hi = (long)edge;
        if (lo >= 0 && lo < (long)p->n_bins) slack[lo] += r->E;
        if (hi >= 0 && hi < (long)p->n_bins) slack[hi] += r->E;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* public scan entry                                                        */
/* ------------------------------------------------------------------------ */
/* The scan with the closest-hit and any-hit queries answered through a CPU
   BVH built by orc_bvh_build (bvh != NULL) instead of brute force; fast != 0
   selects the timing mode (strict pruning, tabulated windows, no parity
   flags).  bvh == NULL is the oracle itself. */
int orc_scan_accel(const float* vertices, uint32_t n_vertices, const uint32_t* triangles, uint32_t n_triangles,
                   const uint16_t* material_ids, const orc_material* materials, uint32_t n_materials,
                   const orc_pose* pose, const orc_params* p, const uint32_t* az_list, uint32_t n_cols, double* image,
                   double* image_masked, double* slack, uint8_t* ray_flags, double* tallies, orc_segment* segs,
                   uint64_t seg_cap, uint64_t* n_segs, uint64_t* counts, int n_threads, const orc_bvh* bvh,
                   int fast) {
  if (p->n_azimuth == 0 || p->rays_per_beam == 0 || p->n_bins == 0 || p->max_bounces == 0) return 1;
  for (uint32_t j = 0; j < n_triangles; ++j) {
    for (int i = 0; i < 3; ++i)
      if (triangles[3 * (size_t)j + i] >= n_vertices) return 2;
    if (material_ids[j] >= n_materials) return 2;
  }
  if (bvh && bvh->wtab && bvh->nm != n_materials) return 2;
  if (bvh && !fast && !bvh->exact) return 4; /* the flags need the grown boxes */
  scene_t s = {vertices, triangles, material_ids, materials, n_vertices, n_triangles, n_materials, bvh,
               bvh ? fast : 0};
  column_t* cols = (column_t*)calloc(n_cols, sizeof(column_t));
  const uint32_t ns = p->rays_per_beam;
  for (uint32_t c = 0; c < n_cols; ++c) {
    cols[c].keep_segs = segs != NULL;
    cols[c].flagged = ray_flags + (size_t)c * ns;
    cols[c].tally = tallies + (size_t)c * ns * 4;
    memset(cols[c].tally, 0, sizeof(double) * 4 * ns);
  }
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int c = 0; c < (int)n_cols; ++c) {
    uint32_t a = az_list ? az_list[c] : (uint32_t)c;
    trace_column(&s, p, pose, a, &cols[c]);
    bin_column(p, &cols[c], image + (size_t)c * p->n_bins,
               image_masked ? image_masked + (size_t)c * p->n_bins : NULL,
               slack ? slack + (size_t)c * p->n_bins : NULL);
  }
  uint64_t ns_out = 0, q = 0, sq = 0, nret = 0;
  for (uint32_t c = 0; c < n_cols; ++c) {
    if (!segs) ns_out += cols[c].n_seg;
    for (size_t i = 0; segs && i < cols[c].n_seg; ++i) {
      if (ns_out < seg_cap) segs[ns_out] = cols[c].seg[i];
      ns_out++;
    }
    q += cols[c].queries;
    sq += cols[c].shadow_queries;
    nret += cols[c].n_ret;
    free(cols[c].seg);
    free(cols[c].ret);
  }
  free(cols);
  if (n_segs) *n_segs = ns_out;
  if (counts) {
    counts[0] = q;
    counts[1] = sq;
    counts[2] = nret;
  }
  return (segs && ns_out > seg_cap) ? 3 : 0;
}

int orc_scan(const float* vertices, uint32_t n_vertices, const uint32_t* triangles, uint32_t n_triangles,
             const uint16_t* material_ids, const orc_material* materials, uint32_t n_materials, const orc_pose* pose,
             const orc_params* p, const uint32_t* az_list, uint32_t n_cols, double* image, double* image_masked,
             double* slack, uint8_t* ray_flags, double* tallies, orc_segment* segs, uint64_t seg_cap,
             uint64_t* n_segs, uint64_t* counts, int n_threads) {
  return orc_scan_accel(vertices, n_vertices, triangles, n_triangles, material_ids, materials, n_materials, pose, p,
                        az_list, n_cols, image, image_masked, slack, ray_flags, tallies, segs, seg_cap, n_segs, counts,
                        n_threads, NULL, 0);
}

/* number of threads an OpenMP region would use */
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Sec. III-C noise and the post pass.                                       */
/*  (1) optional beam pattern across azimuths (circular Gaussian),          */
/*  (2) measurement noise as a Gaussian blur along range (zero padded),     */
/*  (3) additive uniform system and ambient noise.                          */
/* Taps: exp(-j^2 / (2 sigma^2)) for |j| <= ceil(3 sigma), normalised.      */
/* ------------------------------------------------------------------------ */
static int gauss_taps(double sigma, double* w, int max_r) {
  if (!(sigma > 0.0)) {
    w[0] = 1.0;
    return 0;
  }
  int r = (int)ceil(3.0 * sigma);
  if (r > max_r) r = max_r;
  double sum = 0.0;
  for (int j = -r; j <= r; ++j) {
    w[j + r] = exp(-0.5 * (double)j * (double)j / (sigma * sigma));
    sum += w[j + r];
  }
  for (int j = 0; j <= 2 * r; ++j) w[j] /= sum;
  return r;
}

/* Sec. III-C, the Perlin noise model of ambient and system noise: gradient
   noise (Perlin, "Improving noise", SIGGRAPH 2002) over the polar image.  The
   lattice has P = max(1, round(n_az / cell_az)) cells around the circle
   (periodic) and cells of cell_bins bins along range: pixel (a, bin) sits at
   x = a P / n_az, y = bin / cell_bins.  Lattice point (I, J) carries the
   unit gradient of angle 2 pi u, u the uniform of Philox counter
   (scan_id, I, J, purpose) -- purpose 4 for system, 5 for ambient noise.
   The four corner ramps are blended with the fade 6t^5 - 15t^4 + 10t^3; the
   noise n lies in [-1/sqrt(2), 1/sqrt(2)] and is mapped to 1/2 + n/sqrt(2)
   in [0, 1]. */
static double perlin_fade(double t) { return t * t * t * (t * (6.0 * t - 15.0) + 10.0); }

static void perlin_grad(const orc_params* p, uint32_t I, uint32_t J, uint32_t purpose, double g[2]) {
  uint32_t x[4];
  draw(p, I, J, purpose, x);
  double th = 2.0 * M_PI * orc_u24(x[0]);
  g[0] = cos(th);
  g[1] = sin(th);
}

double orc_perlin(const orc_params* p, uint32_t a, uint32_t bin, uint32_t purpose) {
  long P = lround((double)p->n_azimuth / p->noise_cell_az);
  if (P < 1) P = 1;
  double x = (double)a * (double)P / (double)p->n_azimuth;
  double y = (double)bin / p->noise_cell_bins;
  double xf = floor(x), yf = floor(y);
  uint32_t i0 = (uint32_t)xf % (uint32_t)P, i1 = (i0 + 1u) % (uint32_t)P;
  uint32_t j0 = (uint32_t)yf, j1 = j0 + 1u;
  double fx = x - xf, fy = y - yf;
  double g00[2], g10[2], g01[2], g11[2];
  perlin_grad(p, i0, j0, purpose, g00);
  perlin_grad(p, i1, j0, purpose, g10);
  perlin_grad(p, i0, j1, purpose, g01);
  perlin_grad(p, i1, j1, purpose, g11);
  double n00 = g00[0] * fx + g00[1] * fy;
  double n10 = g10[0] * (fx - 1.0) + g10[1] * fy;
  double n01 = g01[0] * fx + g01[1] * (fy - 1.0);
  double n11 = g11[0] * (fx - 1.0) + g11[1] * (fy - 1.0);
  double sx = perlin_fade(fx), sy = perlin_fade(fy);
  double nx0 = n00 + sx * (n10 - n00), nx1 = n01 + sx * (n11 - n01);
  double n = nx0 + sy * (nx1 - nx0);
  return 0.5 + n / sqrt(2.0);
}

/* image: [n_cols][n_bins] for the azimuth indices az_list (NULL = all).  The
   azimuth pattern needs every column and is refused on a subset. */
int orc_post(double* image, const orc_params* p, const uint32_t* az_list, uint32_t n_cols) {
  const uint32_t nb = p->n_bins;
  enum { MAXR = 4096 };
  double* tmp = NULL;
  if (p->az_pattern_sigma > 0.0) {
    if (n_cols != p->n_azimuth || az_list) return 1;
    double* w = (double*)malloc(sizeof(double) * (2 * MAXR + 1));
    int r = gauss_taps(p->az_pattern_sigma, w, MAXR);
    tmp = (double*)calloc((size_t)n_cols * nb, sizeof(double));
    for (uint32_t a = 0; a < n_cols; ++a)
      for (int j = -r; j <= r; ++j) {
        long src = ((long)a + j) % (long)n_cols;
        if (src < 0) src += n_cols;
        for (uint32_t i = 0; i < nb; ++i) tmp[(size_t)a * nb + i] += w[j + r] * image[(size_t)src * nb + i];
      }
    memcpy(image, tmp, sizeof(double) * (size_t)n_cols * nb);
    free(tmp);
    free(w);
  }
  if (p->blur_sigma_bins > 0.0) {
    double* wtab = (double*)malloc(sizeof(double) * (2 * MAXR + 1));
    int r = gauss_taps(p->blur_sigma_bins, wtab, MAXR);
    double* col = (double*)malloc(sizeof(double) * nb);
    for (uint32_t a = 0; a < n_cols; ++a) {
      double* img = image + (size_t)a * nb;
      for (uint32_t i = 0; i < nb; ++i) {
        double acc = 0.0;
        for (int j = -r; j <= r; ++j) {
          long src = (long)i + j;
          if (src < 0 || src >= (long)nb) continue;
          acc += wtab[j + r] * img[src];
        }
        col[i] = acc;
      }
      memcpy(img, col, sizeof(double) * nb);
    }
    free(col);
    free(wtab);
  }
  if (p->flags & ORC_NOISE) {
    for (uint32_t c = 0; c < n_cols; ++c) {
      uint32_t a = az_list ? az_list[c] : c;
      for (uint32_t i = 0; i < nb; ++i) {
        double vs, va;
        if (p->flags & ORC_NOISE_PERLIN) {
          vs = orc_perlin(p, a, i, 4u);
          va = orc_perlin(p, a, i, 5u);
        } else {
          uint32_t xs[4], xa[4];
          draw(p, a, i, 2u, xs);
          draw(p, a, i, 3u, xa);
          vs = orc_u24(xs[0]);
          va = orc_u24(xa[0]);
        }
        image[(size_t)c * nb + i] += p->noise_sys * vs + p->noise_amb * va;
      }
    }
  }
  return 0;
}

/* Sec. III-B: L_E = 10 log10(E_R / E0), E0 = 1 per column, mapped linearly
   from [-cutoff_db, 0] dB to [0, 255] and clamped. */
void orc_db_u8(const double* image, uint64_t n, double cutoff_db, uint8_t* out) {
  for (uint64_t i = 0; i < n; ++i) {
    double e = image[i];
    double v;
    if (!(e > 0.0)) {
      v = 0.0;
    } else {
      double le = 10.0 * log10(e);
      v = 255.0 * (le + cutoff_db) / cutoff_db;
      if (v < 0.0) v = 0.0;
      if (v > 255.0) v = 255.0;
    }
    out[i] = (uint8_t)floor(v + 0.5);
  }
}
