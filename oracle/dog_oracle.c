/*
 * dog_oracle.c -- single-threaded CPU oracle of the DS-PHD/MIB dynamic occupancy grid
 * filter (Nuss et al., "A Random Finite Set Approach for Dynamic Occupancy Grid Maps with
 * Real-Time Application", Sect. VI and Sect. VII).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may load this library.  It shares no code, header, table or constant
 * generator with the CUDA path under paper_1605_02406_b300/; it is written straight
 * from the paper's equations, one plain loop per step, in the paper's order:
 *
 *   a1 particle prediction        Eq. (process), Eq. (particle_persistence), Alg. 1
 *   a2 sort + cell assignment     Alg. 2
 *   a3 predicted occupied mass    Eq. (predExistenceProb) / (DS_particle_sum_pred), Alg. 3
 *   a4 DS mass update + split     Eq. (DS_freespace_pred), (DS_comb), (DS_resulting_masses1/2)
 *   a5 weight normalisation       Eq. (DSupdateParticleWeightsUnnormalized), (DSnormalization),
 *                                 (DSnormalizationfactor), (DSnormalizationfactor2), Alg. 4;
 *      velocity moments           Eq. (mean_x), (var_x), (covar_xy), Alg. 6
 *   a6 newborn particles          Eq. (weights_associated), (weights_unassociated),
 *                                 (assoc_relation), (assoc_sum), Alg. 5
 *   a7 systematic resampling      Eq. (resampledParticleWeights), Alg. 7
 *
 * Compiled twice from this one file:
 *   -DORACLE_F32  "FP32 mirror": IEEE binary32, no contraction (-ffp-contract=off), own
 *                 ln / sincos(2 pi u) / exp from their series definitions, so that every
 *                 decision that floating point turns into an integer (cell index, birth
 *                 slot, resample source) is taken in the kernel's precision.
 *   (default)     FP64: the same steps in binary64 with libm transcendentals.
 * Both modes keep the 64-bit fixed-point weight sums that the method fixes (scale 2^40).
 *
 * Where the paper is silent or ambiguous, the reading taken is marked "reading" at the
 * place it is applied below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORACLE_F32
typedef float real;
#define R(c) c##f
#else
typedef double real;
#define R(c) c
#endif

#define OR_NO_RESAMPLE 0x2u
#define OR_FULL 0x40u /* the PHD/MIB filter of Sect. VI instead of the DS approximation */

typedef struct {
  int32_t width, height;
  float cell_size;
  uint32_t nu, nu_b;
  float p_S, p_B, alpha, sigma_pos, sigma_vel, sigma_birth_vel, sensor_x, sensor_y;
  uint64_t seed;
  uint32_t flags;
} or_params;

typedef struct {
  or_params p;
  int64_t C;
  uint32_t frame;
  /* posterior state */
  real *x, *y, *vx, *vy, *w; /* [nu] */
  real *mF;                  /* [C]  posterior free mass */
  /* measurement grid */
  real *zO, *zF, *pA, *zv, *sgv; /* [C] */
  int has_radar;
  /* per-cell outputs of the last frame */
  real *mO, *rho_p, *rho_b, *pO, *mean_x, *mean_y, *var_x, *var_y, *cov, *mpred, *muA, *muU;
  /* intermediates of the last frame (for parity tests) */
  real *px, *py, *pvx, *pvy, *pw; /* predicted particles, original order [nu] */
  uint32_t *key;                  /* [nu] */
  uint32_t *perm;                 /* [nu] sorted position -> original index */
  uint32_t *cstart, *cend;        /* [C] half-open sorted range, 0/0 when empty */
  uint64_t *S, *A;                /* [C] fixed-point sums of w and g*w */
  real *wn;                       /* [nu] normalised weights in sorted order */
  real *bx, *by, *bvx, *bvy, *bw; /* [nu_b] newborn particles */
  uint32_t *bcell;                /* [nu_b] cell of each newborn slot */
  uint8_t *bassoc;                /* [nu_b] 1 = associated set */
  uint32_t *rsrc;                 /* [nu] resampled source index (joint index space) */
  uint64_t Wq, RC, u;
  /* PHD/MIB filter (OR_FULL): Bernoulli observation per cell and per-cell intermediates */
  real *bz, *bptp, *bpfp, *bpa, *bpc; /* [C] z, p_TP, p_FP, p_A, p_c */
  real *rbp, *fcell;                  /* [C] predicted newborn existence, update factor */
  /* ego motion to apply at the start of the next step (oracle_set_ego_motion) */
  int ego_on;
  real ego_c, ego_s, ego_dx, ego_dy;
  uint8_t *inflag;                  /* [nu] 1 = the predicted particle lies inside the grid */
  /* decisions taken from another run for the next step only (oracle_force_decisions):
   * each particle's cell and in-grid flag, each newborn slot's cell and set, whether any
   * newborn mass existed, whether the frame resampled, and each resampled source */
  int forced;
  uint32_t *fkey, *fbcell, *frsrc;
  uint8_t *fin, *fbassoc;
  int fbirth_mass, fresampled;
} oracle;

/* ------------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11): counter-based, 10 rounds, multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key
 * increments 0x9E3779B9 / 0xBB67AE85 applied before every round after the first.
 * ------------------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

enum { TAG_INIT = 0, TAG_PREDICT = 1, TAG_BIRTH = 2, TAG_RESAMPLE = 3 };

static void draw(const oracle *o, uint32_t elem, uint32_t frame, uint32_t tag, uint32_t r[4]) {
  uint32_t ctr[4] = {elem, frame, tag, 0u};
  uint32_t key[2] = {(uint32_t)o->p.seed, (uint32_t)(o->p.seed >> 32)};
  oracle_philox4x32_10(ctr, key, r);
}

/* uniform on [0,1): top 24 bits; on (0,1]: top 24 bits + 1 ulp of 2^-24 */
static real unif_co(uint32_t r) { return (real)(r >> 8) * R(0x1p-24); }
static real unif_oc(uint32_t r) { return (real)((r >> 8) + 1u) * R(0x1p-24); }

/* ------------------------------------------------------------------------------------
 * Transcendentals.  FP32 mirror: own routines from their textbook series, each Horner
 * step one fused multiply-add (fmaf: a single rounding), every other product and sum
 * rounded separately.  FP64: libm.
 * ------------------------------------------------------------------------------------ */
#ifdef ORACLE_F32
static float bits2f(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t f2bits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* ln(u), u a positive normal float: u = m 2^e, m folded into [sqrt(1/2), sqrt(2)],
 * ln m = 2 atanh(s) with s = (m-1)/(m+1) = 2 s (1 + s^2/3 + s^4/5 + ... + s^10/11),
 * ln u = e ln2_hi + (ln m + e ln2_lo)  (ln2 split so that e*ln2_hi is exact). */
float oracle_ln_f32(float u) {
  uint32_t b = f2bits(u);
  int e = (int)((b >> 23) & 0xffu) - 127;
  float m = bits2f((b & 0x7fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) { m = m * 0.5f; e = e + 1; }
  float f = m - 1.0f;
  float t = 2.0f + f;
  float s = f / t;
  float z = s * s;
  float p = 0x1.745d18p-4f;            /* 1/11 */
  p = fmaf(p, z, 0x1.c71c72p-4f);      /* 1/9 */
  p = fmaf(p, z, 0x1.24924ap-3f);      /* 1/7 */
  p = fmaf(p, z, 0x1.99999ap-3f);      /* 1/5 */
  p = fmaf(p, z, 0x1.555556p-2f);      /* 1/3 */
  p = fmaf(p, z, 1.0f);
  float s2 = s + s;
  float lnm = s2 * p;
  float ef = (float)e;
  float c = fmaf(ef, 0x1.7f7d1cp-20f, lnm);  /* lnm + e * ln2_lo */
  return fmaf(ef, 0x1.62e4p-1f, c);          /* + e * ln2_hi */
}

/* sin and cos of 2 pi u for u = k 2^-24 in [0,1): octant k = floor(8u), t = 8u - k,
 * odd octants use 1 - t; theta = t pi/4 in [0, pi/4]; Taylor series of sin to theta^9
 * and cos to theta^10; the octant's symmetry then picks and signs the pair. */
void oracle_sincos2pi_f32(float u, float *sn, float *cs) {
  float v = u * 8.0f;
  int k = (int)v;
  float t = v - (float)k;
  float tt = (k & 1) ? (1.0f - t) : t;
  float th = tt * 0x1.921fb6p-1f; /* pi/4 */
  float z = th * th;
  float ps = 0x1.71de3ap-19f;               /* 1/9! */
  ps = fmaf(ps, z, -0x1.a01a02p-13f);       /* -1/7! */
  ps = fmaf(ps, z, 0x1.111112p-7f);         /* 1/5! */
  ps = fmaf(ps, z, -0x1.555556p-3f);        /* -1/3! */
  ps = fmaf(ps, z, 1.0f);
  float S = th * ps;
  float pc = -0x1.27e4fcp-22f;              /* -1/10! */
  pc = fmaf(pc, z, 0x1.a01a02p-16f);        /* 1/8! */
  pc = fmaf(pc, z, -0x1.6c16c2p-10f);       /* -1/6! */
  pc = fmaf(pc, z, 0x1.555556p-5f);         /* 1/4! */
  pc = fmaf(pc, z, -0.5f);                  /* -1/2! */
  pc = fmaf(pc, z, 1.0f);
  float Cv = pc;
  switch (k) {
    case 0: *sn = S; *cs = Cv; break;
    case 1: *sn = Cv; *cs = S; break;
    case 2: *sn = Cv; *cs = -S; break;
    case 3: *sn = S; *cs = -Cv; break;
    case 4: *sn = -S; *cs = -Cv; break;
    case 5: *sn = -Cv; *cs = -S; break;
    case 6: *sn = -Cv; *cs = S; break;
    default: *sn = -S; *cs = Cv; break;
  }
}

/* e^x for x <= 0: x = k ln2 + r with k = floor(x/ln2 + 1/2) (Cody-Waite split of ln2),
 * e^r by its Taylor series to r^7, times 2^k assembled in the exponent field.
 * Below -87 the result is flushed to 0. */
float oracle_exp_f32(float x) {
  if (!(x > -87.0f)) return 0.0f;
  float t = fmaf(x, 0x1.715476p+0f, 0.5f); /* x/ln2 + 1/2 */
  float kf = floorf(t);
  int k = (int)kf;
  float r1 = fmaf(-kf, 0x1.62e4p-1f, x);    /* x - k ln2_hi (k ln2_hi exact) */
  float r = fmaf(-kf, 0x1.7f7d1cp-20f, r1); /* - k ln2_lo */
  float p = 0x1.a01a02p-13f;            /* 1/7! */
  p = fmaf(p, r, 0x1.6c16c2p-10f);      /* 1/6! */
  p = fmaf(p, r, 0x1.111112p-7f);       /* 1/5! */
  p = fmaf(p, r, 0x1.555556p-5f);       /* 1/4! */
  p = fmaf(p, r, 0x1.555556p-3f);       /* 1/3! */
  p = fmaf(p, r, 0.5f);                 /* 1/2! */
  p = fmaf(p, r, 1.0f);
  p = fmaf(p, r, 1.0f);
  float sc = bits2f((uint32_t)(k + 127) << 23);
  return p * sc;
}
#define R_LN(u) oracle_ln_f32(u)
#define R_EXP(x) oracle_exp_f32(x)
static void r_sincos2pi(real u, real *s, real *c) { oracle_sincos2pi_f32(u, s, c); }
#define R_SQRT(x) sqrtf(x)
#define R_MIN(a, b) fminf(a, b)
#else
#define R_LN(u) log(u)
#define R_EXP(x) exp(x)
static void r_sincos2pi(real u, real *s, real *c) {
  double a = 6.283185307179586476925 * u; /* 2 pi u */
  *s = sin(a);
  *c = cos(a);
}
#define R_SQRT(x) sqrt(x)
#define R_MIN(a, b) fmin(a, b)
#endif

/* Box-Muller: two independent N(0,1) from two 32-bit draws. */
static void box_muller(uint32_t ra, uint32_t rb, real *n0, real *n1) {
  real u1 = unif_oc(ra);
  real u2 = unif_co(rb);
  real l = R_LN(u1);
  real t = R(-2.0) * l;
  real rad = R_SQRT(t);
  real s, c;
  r_sincos2pi(u2, &s, &c);
  *n0 = rad * c;
  *n1 = rad * s;
}

/* ------------------------------------------------------------------------------------
 * Fixed point.  Weights: unsigned, scale 2^40, truncation (the method's 64-bit
 * fixed-point weight sums and CDF).  Converting back rounds to nearest.
 * ------------------------------------------------------------------------------------ */
static uint64_t q40(real w) { return (w > 0) ? (uint64_t)(w * R(0x1p40)) : 0u; }
static real fx2r(uint64_t S) { return (real)S * R(0x1p-40); }

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------------------ */
static void *zalloc(size_t n) { return calloc(n ? n : 1, 1); }

oracle *oracle_create(const or_params *p) {
  if (p->width <= 0 || p->height <= 0 || p->nu == 0) return NULL;
  oracle *o = (oracle *)zalloc(sizeof(oracle));
  o->p = *p;
  int64_t C = (int64_t)p->width * p->height;
  o->C = C;
  size_t nu = p->nu, nb = p->nu_b;
#define AR(f, n) o->f = zalloc(sizeof(*o->f) * (n))
  AR(x, nu); AR(y, nu); AR(vx, nu); AR(vy, nu); AR(w, nu);
  AR(mF, C);
  AR(zO, C); AR(zF, C); AR(pA, C); AR(zv, C); AR(sgv, C);
  AR(mO, C); AR(rho_p, C); AR(rho_b, C); AR(pO, C); AR(mean_x, C); AR(mean_y, C);
  AR(var_x, C); AR(var_y, C); AR(cov, C); AR(mpred, C); AR(muA, C); AR(muU, C);
  AR(px, nu); AR(py, nu); AR(pvx, nu); AR(pvy, nu); AR(pw, nu);
  AR(key, nu); AR(perm, nu); AR(cstart, C); AR(cend, C); AR(S, C); AR(A, C);
  AR(wn, nu);
  AR(bx, nb); AR(by, nb); AR(bvx, nb); AR(bvy, nb); AR(bw, nb); AR(bcell, nb); AR(bassoc, nb);
  AR(rsrc, nu);
  AR(bz, C); AR(bptp, C); AR(bpfp, C); AR(bpa, C); AR(bpc, C); AR(rbp, C); AR(fcell, C);
  AR(inflag, nu);
  AR(fkey, nu); AR(fin, nu); AR(fbcell, nb); AR(fbassoc, nb); AR(frsrc, nu);
#undef AR
  for (int64_t c = 0; c < C; ++c) o->sgv[c] = 1;
  /* reading: initial state -- particles uniform over the grid, birth-distribution
   * velocities, weight 0; all cells m_O = m_F = 0 (frame 1 is then births only). */
  real gx = (real)p->width * (real)p->cell_size;
  real gy = (real)p->height * (real)p->cell_size;
  real sB = (real)p->sigma_birth_vel;
  for (uint32_t i = 0; i < p->nu; ++i) {
    uint32_t r[4];
    draw(o, i, 0u, TAG_INIT, r);
    o->x[i] = unif_co(r[0]) * gx;
    o->y[i] = unif_co(r[1]) * gy;
    real n0, n1;
    box_muller(r[2], r[3], &n0, &n1);
    o->vx[i] = sB * n0;
    o->vy[i] = sB * n1;
    o->w[i] = 0;
  }
  return o;
}

void oracle_destroy(oracle *o) {
  if (!o) return;
  void *ptrs[] = {o->x, o->y, o->vx, o->vy, o->w, o->mF, o->zO, o->zF, o->pA, o->zv, o->sgv,
                  o->mO, o->rho_p, o->rho_b, o->pO, o->mean_x, o->mean_y, o->var_x, o->var_y,
                  o->cov, o->mpred, o->muA, o->muU, o->px, o->py, o->pvx, o->pvy, o->pw,
                  o->key, o->perm, o->cstart, o->cend, o->S, o->A, o->wn, o->bx, o->by,
                  o->bvx, o->bvy, o->bw, o->bcell, o->bassoc, o->rsrc, o->bz, o->bptp,
                  o->bpfp, o->bpa, o->bpc, o->rbp, o->fcell, o->inflag, o->fkey, o->fin,
                  o->fbcell, o->fbassoc, o->frsrc};
  for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
  free(o);
}

/* Measurement grid (the paper's meas_cell_array, Sect. VII): occupancy BBA per cell,
 * optional association probability and radial-velocity likelihood parameters. */
int oracle_set_measurement_grid(oracle *o, const double *m_occ, const double *m_free,
                                const double *p_A, const double *z_vr, const double *sigma_vr) {
  for (int64_t c = 0; c < o->C; ++c) {
    double a = m_occ[c], b = m_free[c];
    if (!(a >= 0.0 && a <= 1.0 && b >= 0.0 && b <= 1.0 && a + b <= 1.000001)) return -5;
    if (p_A && !(p_A[c] >= 0.0 && p_A[c] <= 1.0)) return -5;
    if (p_A && p_A[c] > 0.0 && !(sigma_vr[c] > 0.0)) return -5;
  }
  o->has_radar = p_A != NULL;
  for (int64_t c = 0; c < o->C; ++c) {
    o->zO[c] = (real)m_occ[c];
    o->zF[c] = (real)m_free[c];
    o->pA[c] = p_A ? (real)p_A[c] : 0;
    o->zv[c] = p_A ? (real)z_vr[c] : 0;
    o->sgv[c] = p_A ? (real)sigma_vr[c] : 1;
  }
  return 0;
}

/* Bernoulli observation of each cell for the PHD/MIB filter (Sect. VI, Bernoulli
 * Observation Process): z = 1 where a measurement occurred; true / false positive
 * probabilities in (0,1); association probability in [0,1]; clutter density p_c > 0
 * (reading: an occupancy-grid detection carries no position inside its cell, so the
 * single-object likelihood is 1 over the cell and p_c is the clutter-to-object ratio). */
int oracle_set_bernoulli_grid(oracle *o, const double *z, const double *p_tp, const double *p_fp,
                              const double *p_a, const double *p_c) {
  for (int64_t c = 0; c < o->C; ++c) {
    if (!(z[c] == 0.0 || z[c] == 1.0)) return -5;
    if (!(p_tp[c] > 0.0 && p_tp[c] < 1.0 && p_fp[c] > 0.0 && p_fp[c] < 1.0)) return -5;
    if (!(p_a[c] >= 0.0 && p_a[c] <= 1.0) || !(p_c[c] > 0.0 && p_c[c] < 3.0e38)) return -5;
  }
  o->has_radar = 0;
  for (int64_t c = 0; c < o->C; ++c) {
    o->bz[c] = (real)z[c];
    o->bptp[c] = (real)p_tp[c];
    o->bpfp[c] = (real)p_fp[c];
    o->bpa[c] = (real)p_a[c];
    o->bpc[c] = (real)p_c[c];
    o->pA[c] = 0;
  }
  return 0;
}

static int cmp_keyidx(const void *a, const void *b) {
  const uint64_t ka = *(const uint64_t *)a, kb = *(const uint64_t *)b;
  return (ka > kb) - (ka < kb);
}

/* Radar spatial likelihood g (reading: Gaussian in the particle's radial velocity as seen
 * from the sensor; the constant factor cancels in the normalisation Eq. DSnormalizationfactor). */
static real radar_g(real sx, real sy, real x, real y, real vx, real vy, real zv, real sg) {
  real dx = x - sx;
  real dy = y - sy;
  real a = dx * dx;
  real b = dy * dy;
  real r2 = a + b;
  real r = R_SQRT(r2);
  real vr = 0;
  if (r > 0) {
    real e = dx * vx;
    real f = dy * vy;
    real num = e + f;
    vr = num / r;
  }
  real dd = vr - zv;
  real d = dd / sg;
  real d2 = d * d;
  real ex = R(-0.5) * d2;
  return R_EXP(ex);
}
static real likelihood(const oracle *o, real x, real y, real vx, real vy, int64_t c) {
  return radar_g((real)o->p.sensor_x, (real)o->p.sensor_y, x, y, vx, vy, o->zv[c], o->sgv[c]);
}

/* smallest q in [0, a] with (q+1) * d > a * b, i.e. floor(a*b/d), d > 0 */
static uint64_t floor_muldiv(uint64_t a, uint64_t b, uint64_t d) {
  return (uint64_t)(((u128)a * b) / d);
}


/* Per-cell mass prediction and update (Alg. 3):
 *   free-mass prediction            Eq. DS_freespace_pred
 *   Dempster's rule on {O, F}       Eq. DS_comb (reading: normalised conjunctive rule,
 *                                   conflict K = mO zF + mF zO; when 1 - K < 1e-6 the
 *                                   predicted BBA is kept)
 *   newborn / persistent split      Eq. DS_resulting_masses1 / 2 (reading: no births
 *                                   where m_z(O) = 0; a zero denominator gives rho_b = 0) */
static void cell_update(real mp, real mF_prev, real zO, real zF, real alpha, real pB,
                        real *mO_out, real *mF_out, real *rb_out, real *rp_out, real *mFp_out) {
  real t = alpha * mF_prev;
  real u = R(1.0) - mp;
  real mFp = R_MIN(t, u);
  real a1 = R(1.0) - mp;
  real mT = a1 - mFp;
  real b1 = R(1.0) - zO;
  real zT = b1 - zF;
  real k1 = mp * zF;
  real k2 = mFp * zO;
  real K = k1 + k2;
  real den = R(1.0) - K;
  real mO, mF;
  if (den < R(1e-6)) {
    mO = mp;
    mF = mFp;
  } else {
    real o1 = mp * zO, o2 = mp * zT, o3 = mT * zO;
    real o12 = o1 + o2;
    real nO = o12 + o3;
    real f1 = mFp * zF, f2 = mFp * zT, f3 = mT * zF;
    real f12 = f1 + f2;
    real nF = f12 + f3;
    mO = nO / den;
    mF = nF / den;
  }
  real rb = 0;
  if (zO > 0) {
    real g = R(1.0) - mp;
    real pb = pB * g;
    real d = mp + pb;
    if (d > 0) {
      real a = mO * pb;
      rb = a / d;
    }
    if (rb > mO) rb = mO;
  }
  *mO_out = mO;
  *mF_out = mF;
  *rb_out = rb;
  *rp_out = mO - rb;
  *mFp_out = mFp;
}

/* Ego-motion compensation (the paper's experiments compensate the vehicle's motion, from
 * speed and yaw rate, in the grid map, Sect. VIII, without saying how).  Reading: the grid
 * is attached to the vehicle with the sensor at q = (sensor_x, sensor_y); since the
 * previous frame the vehicle moved by d = (dx, dy) in the previous grid's axes and turned
 * by theta about q.  Before the next prediction every posterior particle is expressed in
 * the new grid, p' = q + R(-theta)(p - q - d), v' = R(-theta) v, and the posterior free
 * mass of each new cell is that of the old cell under its centre c, q + R(theta)(c - q) + d
 * (0 when that lies outside the old grid).  cos and sin of theta come from binary64 libm,
 * rounded once in the FP32 mirror.  One call applies to one step. */
void oracle_set_ego_motion(oracle *o, float dx, float dy, float dyaw) {
  o->ego_on = (dx != 0.0f || dy != 0.0f || dyaw != 0.0f);
  o->ego_c = (real)cos((double)dyaw);
  o->ego_s = (real)sin((double)dyaw);
  o->ego_dx = (real)dx;
  o->ego_dy = (real)dy;
}

static void apply_ego_motion(oracle *o) {
  const or_params *p = &o->p;
  const int64_t C = o->C;
  const int W = p->width, H = p->height;
  const real qx = (real)p->sensor_x, qy = (real)p->sensor_y, s = (real)p->cell_size;
  const real c = o->ego_c, sn = o->ego_s, dx = o->ego_dx, dy = o->ego_dy;
  for (uint32_t i = 0; i < p->nu; ++i) {
    real ax = o->x[i] - qx;
    real rx = ax - dx;
    real ay = o->y[i] - qy;
    real ry = ay - dy;
    real t1 = c * rx, t2 = sn * ry;
    real t3 = t1 + t2;
    real t4 = c * ry, t5 = sn * rx;
    real t6 = t4 - t5;
    o->x[i] = qx + t3;
    o->y[i] = qy + t6;
    real vx = o->vx[i], vy = o->vy[i];
    real a1 = c * vx, a2 = sn * vy;
    real b1 = c * vy, b2 = sn * vx;
    o->vx[i] = a1 + a2;
    o->vy[i] = b1 - b2;
  }
  real *mF2 = (real *)malloc(sizeof(real) * (size_t)C);
  for (int64_t cell = 0; cell < C; ++cell) {
    int row = (int)(cell / W), col = (int)(cell % W);
    real cx = (real)col + R(0.5);
    real ux0 = cx * s;
    real ux = ux0 - qx;
    real cy = (real)row + R(0.5);
    real uy0 = cy * s;
    real uy = uy0 - qy;
    real e1 = c * ux, e2 = sn * uy;
    real e3 = e1 - e2;
    real e4 = qx + e3;
    real ox = e4 + dx;
    real g1 = sn * ux, g2 = c * uy;
    real g3 = g1 + g2;
    real g4 = qy + g3;
    real oy = g4 + dy;
    real fx = ox / s, fy = oy / s;
    int in = (fx >= 0 && fx < (real)W && fy >= 0 && fy < (real)H);
    mF2[cell] = in ? o->mF[(int64_t)(int)fy * W + (int)fx] : 0;
  }
  memcpy(o->mF, mF2, sizeof(real) * (size_t)C);
  free(mF2);
}

int oracle_step(oracle *o, float dt_f) {
  const or_params *p = &o->p;
  const uint32_t nu = p->nu, nb = p->nu_b;
  const int64_t C = o->C;
  const int W = p->width, H = p->height;
  const uint32_t f = ++o->frame;
  const real T = (real)dt_f, s = (real)p->cell_size;
  const real sp = (real)p->sigma_pos, sv = (real)p->sigma_vel, pS = (real)p->p_S;

  /* ---- a0: ego-motion compensation of the posterior, if set for this step */
  if (o->ego_on) {
    apply_ego_motion(o);
    o->ego_on = 0;
  }

  /* ---- a1: particle prediction (Eq. process with process noise, Eq. particle_persistence) */
  for (uint32_t i = 0; i < nu; ++i) {
    uint32_t r[4];
    draw(o, i, f, TAG_PREDICT, r);
    real n0, n1, n2, n3;
    box_muller(r[0], r[1], &n0, &n1);
    box_muller(r[2], r[3], &n2, &n3);
    real t1 = T * o->vx[i];
    real t2 = o->x[i] + t1;
    real t3 = sp * n0;
    real x = t2 + t3;
    real u1 = T * o->vy[i];
    real u2 = o->y[i] + u1;
    real u3 = sp * n1;
    real y = u2 + u3;
    real a = sv * n2;
    real vx = o->vx[i] + a;
    real b = sv * n3;
    real vy = o->vy[i] + b;
    real w = pS * o->w[i];
    /* reading: cell index col = floor(x/s), row = floor(y/s); a particle outside the grid
     * gets weight 0 (it can no longer be drawn) and the key of the nearest border cell. */
    real fx = x / s, fy = y / s;
    int in = (fx >= 0 && fx < (real)W && fy >= 0 && fy < (real)H);
    int col = !(fx >= 0) ? 0 : (!(fx < (real)W) ? W - 1 : (int)fx);
    int row = !(fy >= 0) ? 0 : (!(fy < (real)H) ? H - 1 : (int)fy);
    uint32_t key = (uint32_t)row * (uint32_t)W + (uint32_t)col;
    if (o->forced) { /* the other run's decision */
      in = o->fin[i];
      key = o->fkey[i];
    }
    if (!in) w = 0;
    o->px[i] = x; o->py[i] = y; o->pvx[i] = vx; o->pvy[i] = vy; o->pw[i] = w;
    o->key[i] = key;
    o->inflag[i] = (uint8_t)in;
  }

  /* ---- a2: sort particles by cell index (stable: ties keep array order) and assign
   * each cell the half-open range of its particles (Alg. 2). */
  uint64_t *ki = (uint64_t *)malloc(sizeof(uint64_t) * nu);
  for (uint32_t i = 0; i < nu; ++i) ki[i] = ((uint64_t)o->key[i] << 32) | i;
  qsort(ki, nu, sizeof(uint64_t), cmp_keyidx);
  for (uint32_t j = 0; j < nu; ++j) o->perm[j] = (uint32_t)ki[j];
  free(ki);
  memset(o->cstart, 0, sizeof(uint32_t) * C);
  memset(o->cend, 0, sizeof(uint32_t) * C);
  for (uint32_t j = 0; j < nu; ++j) {
    uint32_t c = o->key[o->perm[j]];
    if (j == 0 || o->key[o->perm[j - 1]] != c) o->cstart[c] = j;
    if (j == nu - 1 || o->key[o->perm[j + 1]] != c) o->cend[c] = j + 1;
  }

  /* ---- a3: predicted occupied mass = clamped sum of predicted weights in the cell
   * (Eq. predExistenceProb, DS_particle_sum_pred), as an exact fixed-point sum. */
  memset(o->S, 0, sizeof(uint64_t) * C);
  memset(o->A, 0, sizeof(uint64_t) * C);
  for (uint32_t j = 0; j < nu; ++j) {
    uint32_t i = o->perm[j];
    uint32_t c = o->key[i];
    o->S[c] += q40(o->pw[i]);
    if (o->pA[c] > 0) {
      real g = likelihood(o, o->px[i], o->py[i], o->pvx[i], o->pvy[i], c);
      real gw = g * o->pw[i];
      o->A[c] += q40(gw);
    }
  }

  /* ---- a4: occupancy prediction and DS update per cell (Alg. 3) */
  const real alpha = (real)p->alpha, pB = (real)p->p_B;
  const int full = (p->flags & OR_FULL) != 0;
  for (int64_t c = 0; c < C && full; ++c) {
    /* PHD/MIB filter, Sect. VI.  Predicted Bernoulli RFS: persistent existence r_p = the
     * cell's predicted weight sum, truncated to 1 (reading: the weights of a cell whose sum
     * exceeds 1 are scaled to sum 1), newborn existence r_b = p_B (1 - r_p) (Eq.
     * pred_birth_prob).  Update (Eq. updateParticleWeightsUnnormalized, applyNormalization,
     * normalizationCalculation; updateParticleWeightsEmpty) with a likelihood of 1: every
     * particle weight of the cell is multiplied by one factor f; the sums over the cell's
     * persistent and newborn weights in the normaliser are r_p and r_b. */
    real Sr = fx2r(o->S[c]);
    real rp = R_MIN(Sr, R(1.0));
    real omp = R(1.0) - rp;
    real rb = pB * omp;
    real r = rp + rb;
    real omr = R(1.0) - r;
    real ptp = o->bptp[c], pfp = o->bpfp[c];
    real fc;
    if (o->bz[c] != 0) {
      real pa = o->bpa[c], pc = o->bpc[c];
      real q = R(1.0) - pa;
      real q2 = q * pc;
      real gam = pa + q2;                   /* g_A = p_A g + (1 - p_A) p_c, g = 1 */
      real num = ptp * gam;
      real t1 = pfp * pc;
      real t2 = t1 * omr;
      real t3 = num * r;
      real Nz = t2 + t3;
      fc = num / Nz;
    } else {
      real a = R(1.0) - ptp;
      real b = R(1.0) - pfp;
      real t1 = a * r;
      real t2 = b * omr;
      real Ne = t1 + t2;
      fc = a / Ne;
    }
    real rhop = fc * rp;
    real rhob = fc * rb;
    real rpost = rhop + rhob;              /* posterior existence, Eq. occupancyProbParticles */
    o->mpred[c] = rp;
    o->mO[c] = rpost;
    o->mF[c] = R(1.0) - rpost;             /* reading: the free probability 1 - r' */
    o->rho_p[c] = rhop;
    o->rho_b[c] = rhob;
    o->pO[c] = rpost;
    o->muU[c] = (o->S[c] > 0) ? (Sr > R(1.0) ? fc / Sr : fc) : 0;
    o->muA[c] = fc;
    o->rbp[c] = rb;
    o->fcell[c] = fc;
  }
  for (int64_t c = 0; c < C && !full; ++c) {
    real Sr = fx2r(o->S[c]);
    real mp = R_MIN(Sr, R(1.0));           /* Eq. predExistenceProb: min(sum, 1) */
    real mO, mF, rb, rp, mFp;
    cell_update(mp, o->mF[c], o->zO[c], o->zF[c], alpha, pB, &mO, &mF, &rb, &rp, &mFp);
    /* Eq. DSnormalizationfactor2 with the raw (unclamped) predicted sum */
    real muU = (o->S[c] > 0) ? rp / Sr : 0;
    real muA = (o->A[c] > 0) ? rp / fx2r(o->A[c]) : 0;
    o->mpred[c] = mp;
    o->mO[c] = mO;
    o->mF[c] = mF;
    o->rho_b[c] = rb;
    o->rho_p[c] = rp;
    real q = R(1.0) - mO;
    real q2 = q - mF;
    real h = R(0.5) * q2;
    o->pO[c] = mO + h;                     /* pignistic transformation */
    o->muU[c] = muU;
    o->muA[c] = muA;
  }

  /* ---- a5: normalise persistent particle weights (Eq. DSnormalization, Alg. 4) */
  for (uint32_t j = 0; j < nu; ++j) {
    uint32_t i = o->perm[j];
    uint32_t c = o->key[i];
    real w = o->pw[i];
    real wn;
    real pA = (o->A[c] > 0) ? o->pA[c] : 0; /* reading: no likelihood mass -> g ignored */
    if (pA > 0) {
      real g = likelihood(o, o->px[i], o->py[i], o->pvx[i], o->pvy[i], c);
      real t1 = pA * o->muA[c];
      real t2 = t1 * g;
      real t3 = t2 * w;
      real t4 = R(1.0) - pA;
      real t5 = t4 * o->muU[c];
      real t6 = t5 * w;
      wn = t3 + t6;
    } else {
      wn = o->muU[c] * w;
    }
    o->wn[j] = wn;
  }
  /* velocity moments of the persistent posterior particles (Eq. mean_x, var_x, covar_xy),
   * summed in binary64 straight from their definition */
  {
    double *acc = (double *)calloc((size_t)C * 5, sizeof(double));
    for (uint32_t j = 0; j < nu; ++j) {
      uint32_t i = o->perm[j];
      uint32_t c = o->key[i];
      double wn = (double)o->wn[j], vx = (double)o->pvx[i], vy = (double)o->pvy[i];
      acc[5 * c + 0] += wn * vx;
      acc[5 * c + 1] += wn * vy;
      acc[5 * c + 2] += wn * vx * vx;
      acc[5 * c + 3] += wn * vy * vy;
      acc[5 * c + 4] += wn * vx * vy;
    }
    for (int64_t c = 0; c < C; ++c) {
      double rp = (double)o->rho_p[c];
      if (rp > 0) {
        double mx = acc[5 * c] / rp, my = acc[5 * c + 1] / rp;
        double vxx = acc[5 * c + 2] / rp - mx * mx;
        double vyy = acc[5 * c + 3] / rp - my * my;
        o->mean_x[c] = (real)mx;
        o->mean_y[c] = (real)my;
        o->var_x[c] = (real)(vxx > 0 ? vxx : 0);
        o->var_y[c] = (real)(vyy > 0 ? vyy : 0);
        o->cov[c] = (real)(acc[5 * c + 4] / rp - mx * my);
      } else {
        o->mean_x[c] = o->mean_y[c] = o->var_x[c] = o->var_y[c] = o->cov[c] = 0;
      }
    }
    free(acc);
  }

  /* ---- a6: newborn particles (Alg. 5) */
  /* newborn slots follow the posterior newborn mass (DS) or, in the PHD/MIB filter, the
   * predicted newborn existence (Sect. VI: births are sampled in the prediction) */
  const real *bmass = full ? o->rbp : o->rho_b;
  uint64_t RC = 0;
  for (int64_t c = 0; c < C; ++c) RC += q40(bmass[c]);
  o->RC = RC;
  const real sB = (real)p->sigma_birth_vel;
  if (o->forced) {
    /* the other run's newborn slots: the same cells and sets, weights from this run's
     * newborn masses with those counts (Eq. weights_associated / unassociated) */
    uint32_t *cnt = (uint32_t *)calloc((size_t)C, sizeof(uint32_t));
    uint32_t *cntA = (uint32_t *)calloc((size_t)C, sizeof(uint32_t));
    for (uint32_t b = 0; b < nb; ++b) {
      cnt[o->fbcell[b]] += 1;
      cntA[o->fbcell[b]] += o->fbassoc[b];
    }
    for (uint32_t b = 0; b < nb; ++b) {
      uint32_t c = o->fbcell[b];
      o->bcell[b] = c;
      o->bassoc[b] = o->fbassoc[b];
      real rb = bmass[c], pA = o->pA[c], wb;
      uint32_t n = cnt[c], nA = cntA[c], nUA = n - nA;
      if (!o->fbirth_mass) wb = 0;
      else if (full) { real a = rb / (real)n; wb = o->fcell[c] * a; }
      else if (nA > 0 && nUA > 0) {
        if (o->fbassoc[b]) { real a = pA * rb; wb = a / (real)nA; }
        else { real q = R(1.0) - pA; real bb = q * rb; wb = bb / (real)nUA; }
      } else wb = rb / (real)n;
      o->bw[b] = wb;
    }
    free(cnt);
    free(cntA);
  } else if (RC == 0) {
    /* reading: no birth mass anywhere -- slots get weight 0 and cell (slot mod C) */
    for (uint32_t b = 0; b < nb; ++b) {
      o->bcell[b] = (uint32_t)(b % (uint64_t)C);
      o->bassoc[b] = 0;
      o->bw[b] = 0;
    }
  } else {
    /* reading: the scan of born masses normalised to nu_b -- cell c owns the slots
     * [floor(nu_b R_{c-1} / R_C), floor(nu_b R_c / R_C)) */
    uint64_t Rprev = 0;
    for (int64_t c = 0; c < C; ++c) {
      uint64_t qb = q40(bmass[c]);
      if (qb == 0) continue;
      uint64_t Rc = Rprev + qb;
      uint32_t lo = (uint32_t)floor_muldiv(nb, Rprev, RC);
      uint32_t hi = (uint32_t)floor_muldiv(nb, Rc, RC);
      Rprev = Rc;
      uint32_t n = hi - lo;
      if (n == 0) continue;
      /* Eq. assoc_relation / assoc_sum; reading: nu_A = round(n p_A), an empty set hands
       * its share of rho_b to the other set */
      real pA = o->pA[c];
      real tn = (real)n * pA;
      tn = tn + R(0.5);
      uint32_t nA = (uint32_t)tn;
      if (nA > n) nA = n;
      uint32_t nUA = n - nA;
      real rb = bmass[c];
      real wA = 0, wUA = 0;
      if (full) {
        /* Eq. predExistenceProbParticlesBorn: r_b / n, then the cell's update factor */
        real a = rb / (real)n;
        wUA = o->fcell[c] * a;
        nA = 0;
      } else if (nA > 0 && nUA > 0) {
        real a = pA * rb;
        wA = a / (real)nA;                  /* Eq. weights_associated */
        real b = R(1.0) - pA;
        real bb = b * rb;
        wUA = bb / (real)nUA;               /* Eq. weights_unassociated */
      } else if (nA > 0) {
        wA = rb / (real)nA;
      } else {
        wUA = rb / (real)nUA;
      }
      for (uint32_t k = 0; k < n; ++k) {
        uint32_t b = lo + k;
        o->bcell[b] = (uint32_t)c;
        o->bassoc[b] = k < nA;
        o->bw[b] = (k < nA) ? wA : wUA;
      }
    }
  }
  /* newborn states: position uniform in the cell; velocity from the birth distribution
   * N(0, sigma_B^2 I) (unassociated, Eq. DSbirth_particle_sampling) or, associated,
   * radial component from the measured radial velocity (Eq. DSbirth_particle_samplingA) */
  for (uint32_t b = 0; b < nb; ++b) {
    uint32_t c = o->bcell[b];
    uint32_t r[4];
    draw(o, b, f, TAG_BIRTH, r);
    real col = (real)(c % (uint32_t)W), row = (real)(c / (uint32_t)W);
    real ux = unif_co(r[0]), uy = unif_co(r[1]);
    real xa = col + ux;
    real x = xa * s;
    real ya = row + uy;
    real y = ya * s;
    real n0, n1;
    box_muller(r[2], r[3], &n0, &n1);
    real vx, vy;
    if (o->bassoc[b]) {
      real dx = x - (real)p->sensor_x, dy = y - (real)p->sensor_y;
      real a = dx * dx;
      real bb = dy * dy;
      real r2 = a + bb;
      real rr = R_SQRT(r2);
      real ex = 1, ey = 0;
      if (rr > 0) {
        ex = dx / rr;
        ey = dy / rr;
      }
      real t = o->sgv[c] * n0;
      real vr = o->zv[c] + t;
      real vt = sB * n1;
      real e1 = vr * ex, e2 = vt * ey;
      vx = e1 - e2;
      real e3 = vr * ey, e4 = vt * ex;
      vy = e3 + e4;
    } else {
      vx = sB * n0;
      vy = sB * n1;
    }
    o->bx[b] = x; o->by[b] = y; o->bvx[b] = vx; o->bvy[b] = vy;
  }

  /* ---- a7: systematic resampling of nu particles from the joint set (Alg. 7) */
  uint64_t Wq = 0;
  for (uint32_t j = 0; j < nu; ++j) Wq += q40(o->wn[j]);
  for (uint32_t b = 0; b < nb; ++b) Wq += q40(o->bw[b]);
  o->Wq = Wq;
  real *nx = (real *)malloc(sizeof(real) * nu), *ny = (real *)malloc(sizeof(real) * nu);
  real *nvx = (real *)malloc(sizeof(real) * nu), *nvy = (real *)malloc(sizeof(real) * nu);
  real *nw = (real *)malloc(sizeof(real) * nu);
  const int resample = o->forced ? o->fresampled : !((p->flags & OR_NO_RESAMPLE) || Wq == 0);
  if (!resample) {
    /* reading: with no weight left (or resampling switched off) the persistent particles
     * carry over in sorted order with their own normalised weights */
    for (uint32_t i = 0; i < nu; ++i) {
      uint32_t s0 = o->perm[i];
      nx[i] = o->px[s0]; ny[i] = o->py[s0]; nvx[i] = o->pvx[s0]; nvy[i] = o->pvy[s0];
      nw[i] = o->wn[i];
      o->rsrc[i] = i;
    }
    o->u = 0;
  } else {
    uint32_t r[4];
    draw(o, 0u, f, TAG_RESAMPLE, r);
    uint64_t r64 = ((uint64_t)r[0] << 32) | r[1];
    uint64_t u = (uint64_t)(((u128)r64 * Wq) >> 64); /* uniform offset in [0, Wq) */
    o->u = u;
    /* the resampled weight: total posterior weight shared equally (Eq. resampledParticleWeights) */
    real wnew = (real)(((double)Wq * 0x1p-40) / (double)nu);
    /* output i takes the first source whose inclusive CDF exceeds floor((i Wq + u) / nu);
     * sources are the persistent particles in sorted order, then the newborn slots */
    uint64_t Q = 0;
    uint32_t j = 0;
    const uint32_t ntot = nu + nb;
    Q = q40(o->wn[0]);
    for (uint32_t i = 0; i < nu; ++i) {
      if (o->forced) {
        j = o->frsrc[i];  /* the other run's source */
      } else {
        uint64_t P = (uint64_t)(((u128)i * Wq + u) / nu);
        while (!(Q > P)) {
          ++j;
          if (j >= ntot) return -9; /* cannot happen: P < Wq */
          Q += (j < nu) ? q40(o->wn[j]) : q40(o->bw[j - nu]);
        }
      }
      o->rsrc[i] = j;
      if (j < nu) {
        uint32_t s0 = o->perm[j];
        nx[i] = o->px[s0]; ny[i] = o->py[s0]; nvx[i] = o->pvx[s0]; nvy[i] = o->pvy[s0];
      } else {
        uint32_t b = j - nu;
        nx[i] = o->bx[b]; ny[i] = o->by[b]; nvx[i] = o->bvx[b]; nvy[i] = o->bvy[b];
      }
      nw[i] = wnew;
    }
  }
  memcpy(o->x, nx, sizeof(real) * nu); memcpy(o->y, ny, sizeof(real) * nu);
  memcpy(o->vx, nvx, sizeof(real) * nu); memcpy(o->vy, nvy, sizeof(real) * nu);
  memcpy(o->w, nw, sizeof(real) * nu);
  free(nx); free(ny); free(nvx); free(nvy); free(nw);
  o->forced = 0;
  return 0;
}

/* Decisions for the next step taken from another run of the same filter (for measuring the
 * arithmetic error of one precision against another on the same Monte Carlo run): each
 * predicted particle's cell index and in-grid flag [nu], each newborn slot's cell and set
 * [nu_b], whether any newborn mass existed, whether the frame resampled and each posterior
 * particle's joint source [nu].  Every real-valued quantity is still computed here. */
void oracle_force_decisions(oracle *o, const uint32_t *key, const uint8_t *in, const uint32_t *bcell,
                            const uint8_t *bassoc, int birth_mass, int resampled, const uint32_t *rsrc) {
  memcpy(o->fkey, key, 4 * (size_t)o->p.nu);
  memcpy(o->fin, in, (size_t)o->p.nu);
  memcpy(o->fbcell, bcell, 4 * (size_t)o->p.nu_b);
  memcpy(o->fbassoc, bassoc, (size_t)o->p.nu_b);
  memcpy(o->frsrc, rsrc, 4 * (size_t)o->p.nu);
  o->fbirth_mass = birth_mass;
  o->fresampled = resampled;
  o->forced = 1;
}

/* ---- accessors (binary64 in and out for both modes; exact for the FP32 mirror) ------- */
static void put(double *dst, const real *src, size_t n) {
  if (!dst) return;
  for (size_t k = 0; k < n; ++k) dst[k] = (double)src[k];
}
static void get(real *dst, const double *src, size_t n) {
  for (size_t k = 0; k < n; ++k) dst[k] = (real)src[k];
}

/* which: 0 m_occ 1 m_free 2 rho_p 3 rho_b 4 p_occ 5 mean_vx 6 mean_vy 7 var_vx 8 var_vy
 * 9 cov_vxy 10 m_occ_pred 11 mu_A 12 mu_UA */
int oracle_get_cell_array(const oracle *o, int which, double *out) {
  const real *src[] = {o->mO, o->mF, o->rho_p, o->rho_b, o->pO, o->mean_x, o->mean_y,
                       o->var_x, o->var_y, o->cov, o->mpred, o->muA, o->muU};
  if (which < 0 || which > 12) return -1;
  put(out, src[which], (size_t)o->C);
  return 0;
}

/* which: 0..4 predicted x,y,vx,vy,w [nu]; 5 normalised weights (sorted) [nu];
 * 6..10 newborn x,y,vx,vy,w [nu_b] */
int oracle_get_particle_array(const oracle *o, int which, double *out) {
  switch (which) {
    case 0: put(out, o->px, o->p.nu); break;
    case 1: put(out, o->py, o->p.nu); break;
    case 2: put(out, o->pvx, o->p.nu); break;
    case 3: put(out, o->pvy, o->p.nu); break;
    case 4: put(out, o->pw, o->p.nu); break;
    case 5: put(out, o->wn, o->p.nu); break;
    case 6: put(out, o->bx, o->p.nu_b); break;
    case 7: put(out, o->by, o->p.nu_b); break;
    case 8: put(out, o->bvx, o->p.nu_b); break;
    case 9: put(out, o->bvy, o->p.nu_b); break;
    case 10: put(out, o->bw, o->p.nu_b); break;
    default: return -1;
  }
  return 0;
}

/* which: 0 key [nu] 1 perm [nu] 2 cell_start [C] 3 cell_end [C] 4 newborn cell [nu_b]
 * 5 newborn associated flag [nu_b] 6 resample source [nu] 7 in-grid flag [nu] */
int oracle_get_index_array(const oracle *o, int which, uint32_t *out) {
  switch (which) {
    case 0: memcpy(out, o->key, 4 * (size_t)o->p.nu); break;
    case 1: memcpy(out, o->perm, 4 * (size_t)o->p.nu); break;
    case 2: memcpy(out, o->cstart, 4 * (size_t)o->C); break;
    case 3: memcpy(out, o->cend, 4 * (size_t)o->C); break;
    case 4: memcpy(out, o->bcell, 4 * (size_t)o->p.nu_b); break;
    case 5: for (uint32_t b = 0; b < o->p.nu_b; ++b) out[b] = o->bassoc[b]; break;
    case 6: memcpy(out, o->rsrc, 4 * (size_t)o->p.nu); break;
    case 7: for (uint32_t i = 0; i < o->p.nu; ++i) out[i] = o->inflag[i]; break;
    default: return -1;
  }
  return 0;
}

/* which: 0 S [C] 1 A [C]; scalars via oracle_get_scalars */
int oracle_get_fixed_array(const oracle *o, int which, uint64_t *out) {
  if (which == 0) memcpy(out, o->S, 8 * (size_t)o->C);
  else if (which == 1) memcpy(out, o->A, 8 * (size_t)o->C);
  else return -1;
  return 0;
}

void oracle_get_scalars(const oracle *o, uint64_t *out /* [4]: frame, Wq, RC, u */) {
  out[0] = o->frame; out[1] = o->Wq; out[2] = o->RC; out[3] = o->u;
}

/* posterior state: particles x,y,vx,vy,w [nu], free mass [C], frame counter */
void oracle_get_state(const oracle *o, double *x, double *y, double *vx, double *vy, double *w,
                      double *m_free, uint32_t *frame) {
  put(x, o->x, o->p.nu); put(y, o->y, o->p.nu); put(vx, o->vx, o->p.nu);
  put(vy, o->vy, o->p.nu); put(w, o->w, o->p.nu); put(m_free, o->mF, (size_t)o->C);
  if (frame) *frame = o->frame;
}

int oracle_set_state(oracle *o, const double *x, const double *y, const double *vx,
                     const double *vy, const double *w, const double *m_free, uint32_t frame) {
  get(o->x, x, o->p.nu); get(o->y, y, o->p.nu); get(o->vx, vx, o->p.nu);
  get(o->vy, vy, o->p.nu); get(o->w, w, o->p.nu); get(o->mF, m_free, (size_t)o->C);
  o->frame = frame;
  return 0;
}

/* direct access to the per-cell update for unit pins (Dempster, split) */
void oracle_cell_update(double m_pred, double m_free_prev, double zO, double zF, double alpha,
                        double pB, double out[5] /* mO, mF, rho_b, rho_p, mF_pred */) {
  real mO, mF, rb, rp, mFp;
  cell_update((real)m_pred, (real)m_free_prev, (real)zO, (real)zF, (real)alpha, (real)pB,
              &mO, &mF, &rb, &rp, &mFp);
  out[0] = mO; out[1] = mF; out[2] = rb; out[3] = rp;
  out[4] = mFp;
}

/* exposed for the pins of the radar likelihood (the mode's arithmetic, inputs rounded to it) */
double oracle_radar_likelihood(double sensor_x, double sensor_y, double x, double y, double vx,
                               double vy, double z_vr, double sigma_vr) {
  return (double)radar_g((real)(float)sensor_x, (real)(float)sensor_y, (real)x, (real)y, (real)vx,
                         (real)vy, (real)z_vr, (real)sigma_vr);
}

/* exposed for the statistical pins of the noise generator */
void oracle_box_muller(uint32_t ra, uint32_t rb, float out[2]) {
  real n0, n1;
  box_muller(ra, rb, &n0, &n1);
  out[0] = (float)n0;
  out[1] = (float)n1;
}
