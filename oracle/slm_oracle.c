/*
 * CPU oracle for SLM split search with particle swarm optimisation
 * (arXiv 2208.07023). TEST INFRASTRUCTURE ONLY: the tests, the smoke check and
 * the benchmark's CPU baseline call it; the product path never does.
 *
 * Plain, slow and sequential by design; the only parallelism is one OpenMP
 * loop over particles, whose evaluations are independent (Sec. IV).
 *
 * What each part follows:
 *   projection f(a) = a^T x ............ Sec. II-A, Eq. (1)
 *   split sets a^T x >= t_b / < t_b ...... Sec. II-A, Eqs. (3)-(4)
 *   threshold search over split points .. Sec. II-A (DFT) and Sec. IV: every
 *        candidate split of a projected 1D subspace is scored and the minimum
 *        kept. The paper gives no bin rule; this oracle uses B uniform bins on
 *        [zmin, zmax] and the B-1 interior bin edges as candidates.
 *   swarm update ......................... Sec. III-A, Eq. (pso-1); the
 *        position is advanced with the NEW velocity (Alg. 1 "Update V_i and
 *        X_i"); r1, r2 are drawn per particle, dimension and iteration.
 *   pbest / gbest ........................ Algorithm 1: strict "<".
 *   tree growth .......................... Algorithm 2 and Sec. II-A (stop
 *        when pure or too small; majority vote in leaves).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp (no fused multiply-add beyond the
 * explicit fmaf of the mirror projection).
 */
#include "slm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, restated from Salmon, Moraes, Dror and Shaw, "Parallel     */
/* random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64  */
/* multiplies with a Weyl-sequence key schedule.                            */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(M0, c0, &hi0, &lo0);
    mulhilo32(M1, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 24 high bits of a 32-bit draw scaled to [0, 1): exact in float. */
static float u01(uint32_t r) { return (float)(r >> 8) * (1.0f / 16777216.0f); }

static void seed_key(uint64_t seed, uint32_t key[2]) {
  key[0] = (uint32_t)seed;
  key[1] = (uint32_t)(seed >> 32);
}

/* Counter of a swarm draw: (node uid, iteration, particle, j/4 | purpose<<24),
 * output lane j mod 4. */
void ora_swarm_uniforms(uint64_t seed, uint32_t node_uid, uint32_t t,
                        int32_t n_particles, int32_t d, int32_t purpose,
                        float* u) {
  uint32_t key[2];
  seed_key(seed, key);
  for (int32_t i = 0; i < n_particles; ++i) {
    for (int32_t j = 0; j < d; ++j) {
      uint32_t ctr[4] = {node_uid, t, (uint32_t)i,
                         ((uint32_t)j >> 2) | ((uint32_t)purpose << 24)};
      uint32_t r[4];
      ora_philox4x32_10(ctr, key, r);
      u[(int64_t)i * d + j] = u01(r[j & 3]);
    }
  }
}

/* Draw k of tree t: counter (t, k/4, 0, purpose<<24), lane k mod 4; the
 * sample is floor(r * n / 2^32). */
void ora_bootstrap(uint64_t seed, uint32_t tree_id, int64_t n, uint32_t* w) {
  uint32_t key[2];
  seed_key(seed, key);
  for (int64_t s = 0; s < n; ++s) w[s] = 0;
  for (int64_t k = 0; k < n; ++k) {
    uint32_t ctr[4] = {tree_id, (uint32_t)(k >> 2), 0u,
                       (uint32_t)ORA_PURPOSE_BOOTSTRAP << 24};
    uint32_t r[4];
    ora_philox4x32_10(ctr, key, r);
    uint64_t s = ((uint64_t)r[k & 3] * (uint64_t)n) >> 32;
    w[s] += 1u;
  }
}

/* ------------------------------------------------------------------------ */
/* Swarm update, Eq. (pso-1):                                               */
/*   v <- omega v + c1 r1 (pB - x) + c2 r2 (gB - x);  x <- x + v             */
/* evaluated left to right, one rounding per operation.                     */

void ora_pso_step(const ora_params* p, int32_t P, int32_t d, double* x,
                  double* v, const double* pbest, const double* gbest,
                  const double* r1, const double* r2) {
  for (int32_t i = 0; i < P; ++i) {
    for (int32_t j = 0; j < d; ++j) {
      int64_t e = (int64_t)i * d + j;
      if (p->precision != ORA_F64) {
        float xv = (float)x[e], vv = (float)v[e];
        float inertia = p->inertia * vv;
        float cog = (p->c1 * (float)r1[e]) * ((float)pbest[e] - xv);
        float soc = (p->c2 * (float)r2[e]) * ((float)gbest[j] - xv);
        float vn = (inertia + cog) + soc;
        v[e] = vn;
        x[e] = xv + vn;
      } else {
        double inertia = (double)p->inertia * v[e];
        double cog = ((double)p->c1 * r1[e]) * (pbest[e] - x[e]);
        double soc = ((double)p->c2 * r2[e]) * (gbest[j] - x[e]);
        double vn = (inertia + cog) + soc;
        v[e] = vn;
        x[e] = x[e] + vn;
      }
    }
  }
}

/* Fuzzy memberships of the evolutionary factor in the four states. */
static float apso_mu(int state, float f) {
  switch (state) {
    case ORA_APSO_EXPLORE:
      if (f <= 0.4f) return 0.0f;
      if (f <= 0.6f) return 5.0f * f - 2.0f;
      if (f <= 0.7f) return 1.0f;
      if (f <= 0.8f) return -10.0f * f + 8.0f;
      return 0.0f;
    case ORA_APSO_EXPLOIT:
      if (f <= 0.2f) return 0.0f;
      if (f <= 0.3f) return 10.0f * f - 2.0f;
      if (f <= 0.4f) return 1.0f;
      if (f <= 0.6f) return -5.0f * f + 3.0f;
      return 0.0f;
    case ORA_APSO_CONVERGE:
      if (f <= 0.1f) return 1.0f;
      if (f <= 0.3f) return -5.0f * f + 1.5f;
      return 0.0f;
    default:
      if (f <= 0.7f) return 0.0f;
      if (f <= 0.9f) return 5.0f * f - 3.5f;
      return 1.0f;
  }
}

static float clamp_c(float c) { return c < 1.5f ? 1.5f : c > 2.5f ? 2.5f : c; }

void ora_apso_step(int32_t P, int32_t d, const double* x, int32_t gpart, int32_t prev_state,
                   float c1, float c2, float delta, ora_apso* out) {
  float dmin = 0.0f, dmax = 0.0f, dg = 0.0f;
  for (int32_t i = 0; i < P; ++i) {
    float acc = 0.0f;
    for (int32_t j = 0; j < P; ++j) {
      if (j == i) continue;
      float s2 = 0.0f;
      for (int32_t k = 0; k < d; ++k) {
        const float diff = (float)x[(int64_t)i * d + k] - (float)x[(int64_t)j * d + k];
        s2 = fmaf(diff, diff, s2);
      }
      acc = acc + sqrtf(s2);
    }
    const float di = P > 1 ? acc / (float)(P - 1) : 0.0f;
    if (i == 0 || di < dmin) dmin = di;
    if (i == 0 || di > dmax) dmax = di;
    if (i == gpart) dg = di;
  }
  const float f = dmax > dmin ? (dg - dmin) / (dmax - dmin) : 0.0f;
  int cand[4], nc = 0;
  float mu[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  for (int sidx = 1; sidx <= 4; ++sidx) {
    mu[sidx] = apso_mu(sidx, f);
    if (mu[sidx] > 0.0f) cand[nc++] = sidx;
  }
  int state = cand[0];
  if (nc > 1) {
    const int next = prev_state % 4 + 1;
    int has_prev = 0, has_next = 0;
    for (int q = 0; q < nc; ++q) {
      has_prev |= cand[q] == prev_state;
      has_next |= cand[q] == next;
    }
    if (has_prev)
      state = prev_state;
    else if (has_next)
      state = next;
    else
      for (int q = 1; q < nc; ++q)
        if (mu[cand[q]] > mu[state]) state = cand[q];
  }
  const float h = 0.5f * delta;
  switch (state) {
    case ORA_APSO_EXPLORE: c1 = c1 + delta; c2 = c2 - delta; break;
    case ORA_APSO_EXPLOIT: c1 = c1 + h; c2 = c2 - h; break;
    case ORA_APSO_CONVERGE: c1 = c1 + h; c2 = c2 + h; break;
    default: c1 = c1 - delta; c2 = c2 + delta; break;
  }
  c1 = clamp_c(c1);
  c2 = clamp_c(c2);
  const float sum = c1 + c2;
  if (sum > 4.0f) {
    c1 = (4.0f * c1) / sum;
    c2 = (4.0f * c2) / sum;
  }
  out->f = f;
  out->state = state;
  out->c1 = c1;
  out->c2 = c2;
  out->w = (float)(1.0 / (1.0 + 1.5 * exp(-2.6 * (double)f)));
}

/* ------------------------------------------------------------------------ */
/* Scoring one projection vector on one node.                               */

static double xlogx(double c) { return c > 0.0 ? c * log(c) : 0.0; }

#define NEAR_TIE_REL 1e-12

static int near_tie(double a, double b) {
  if (a == b || !isfinite(a) || !isfinite(b)) return 0;
  double m = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
  return fabs(a - b) <= NEAR_TIE_REL * m;
}

/* Is candidate a strictly better (lower loss) than b? Gini compares the exact
 * rationals Q = q_num/q_den (larger Q = lower loss); the others compare loss. */
static int better(int criterion, int a_valid, double a_loss, uint64_t a_num,
                  uint64_t a_den, int b_valid, double b_loss, uint64_t b_num,
                  uint64_t b_den) {
  if (!a_valid) return 0;
  if (!b_valid) return 1;
  if (criterion == ORA_GINI) {
    unsigned __int128 lhs = (unsigned __int128)a_num * b_den;
    unsigned __int128 rhs = (unsigned __int128)b_num * a_den;
    return lhs > rhs;
  }
  return a_loss < b_loss;
}

/* Rounds a float to the nearest bfloat16 (8 significant bits), ties to even:
 * add half of the dropped 16 bits (minus one unless the kept part is odd) and
 * truncate. Infinities pass; NaNs stay NaN. */
static float bf16_round(float f) {
  uint32_t u;
  memcpy(&u, &f, sizeof(u));
  if ((u & 0x7f800000u) == 0x7f800000u) {
    if (u & 0x007fffffu) u |= 0x00400000u; /* keep a NaN a NaN */
  } else {
    u += 0x7fffu + ((u >> 16) & 1u);
  }
  u &= 0xffff0000u;
  memcpy(&f, &u, sizeof(f));
  return f;
}

void ora_bf16_round(const float* in, float* out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) out[i] = bf16_round(in[i]);
}

/* Projection arithmetic of one scoring pass. */
enum { PROJ_F64 = 0, PROJ_F32 = 1, PROJ_BF16 = 2 };

/* Position of the lowest set bit of a finite non-zero double. */
static int lsb_exponent(double t) {
  int e;
  double m = frexp(fabs(t), &e); /* t = m 2^e, m in [0.5, 1) */
  uint64_t mi = (uint64_t)ldexp(m, 53);
  int tz = 0;
  while (!(mi & 1u)) {
    mi >>= 1;
    ++tz;
  }
  return e - 53 + tz;
}

/* Histogram over (bin, class) or (bin; weight, sum y, sum y^2), then the
 * threshold scan over the B-1 interior edges (left = bins < b). */
static void score_bins_into(const ora_params* p, const int32_t* labels,
                            const float* y, const int32_t* idx,
                            const uint32_t* wts, int64_t n_idx,
                            const int32_t* bins, ora_eval* out, uint64_t* cnt,
                            double* msum, double* msq, int* tie) {
  const int B = p->n_bins;
  const int K = p->n_classes;
  out->valid = 0;
  out->bin = -1;
  out->loss = INFINITY;
  out->q_num = out->q_den = 0;
  out->n_left = out->n_right = 0.0;
  if (p->criterion == ORA_MSE) {
    memset(cnt, 0, sizeof(uint64_t) * B);
    memset(msum, 0, sizeof(double) * B);
    memset(msq, 0, sizeof(double) * B);
    for (int64_t s = 0; s < n_idx; ++s) {
      uint32_t w = wts ? wts[s] : 1u;
      double ys = (double)y[idx[s]];
      cnt[bins[s]] += w;
      msum[bins[s]] += (double)w * ys;
      msq[bins[s]] += (double)w * ys * ys;
    }
  } else {
    memset(cnt, 0, sizeof(uint64_t) * (size_t)B * K);
    for (int64_t s = 0; s < n_idx; ++s) {
      uint32_t w = wts ? wts[s] : 1u;
      cnt[(int64_t)bins[s] * K + labels[idx[s]]] += w;
    }
  }

  if (p->criterion == ORA_MSE) {
    uint64_t ntot = 0;
    double stot = 0.0, qtot = 0.0;
    for (int b = 0; b < B; ++b) {
      ntot += cnt[b];
      stot += msum[b];
      qtot += msq[b];
    }
    uint64_t nl = 0;
    double sl = 0.0, ql = 0.0;
    for (int b = 1; b < B; ++b) {
      nl += cnt[b - 1];
      sl += msum[b - 1];
      ql += msq[b - 1];
      uint64_t nr = ntot - nl;
      if (nl < (uint64_t)p->min_leaf || nr < (uint64_t)p->min_leaf) continue;
      double sr = stot - sl, qr = qtot - ql;
      double sse_l = ql - sl * sl / (double)nl;
      double sse_r = qr - sr * sr / (double)nr;
      double loss = (sse_l + sse_r) / (double)ntot;
      if (out->valid && near_tie(loss, out->loss)) *tie = 1;
      if (!out->valid || loss < out->loss) {
        out->valid = 1;
        out->bin = b;
        out->loss = loss;
        out->n_left = (double)nl;
        out->n_right = (double)nr;
      }
    }
    return;
  }

  uint64_t tot[64];
  uint64_t left[64];
  uint64_t ntot = 0;
  for (int k = 0; k < K; ++k) {
    tot[k] = 0;
    left[k] = 0;
  }
  for (int b = 0; b < B; ++b)
    for (int k = 0; k < K; ++k) tot[k] += cnt[(int64_t)b * K + k];
  for (int k = 0; k < K; ++k) ntot += tot[k];

  for (int b = 1; b < B; ++b) {
    for (int k = 0; k < K; ++k) left[k] += cnt[(int64_t)(b - 1) * K + k];
    uint64_t nl = 0;
    for (int k = 0; k < K; ++k) nl += left[k];
    uint64_t nr = ntot - nl;
    if (nl < (uint64_t)p->min_leaf || nr < (uint64_t)p->min_leaf) continue;
    if (p->criterion == ORA_GINI) {
      /* n * Gini_w = n - (S_L/n_L + S_R/n_R), S = sum_k n_k^2.
       * Q = (S_L n_R + S_R n_L) / (n_L n_R); lower loss <=> larger Q. */
      uint64_t sl = 0, sr = 0;
      for (int k = 0; k < K; ++k) {
        uint64_t r = tot[k] - left[k];
        sl += left[k] * left[k];
        sr += r * r;
      }
      uint64_t num = sl * nr + sr * nl;
      uint64_t den = nl * nr;
      uint64_t nden = ntot * den;
      double loss = (double)(nden - num) / (double)nden;
      if (better(ORA_GINI, 1, loss, num, den, out->valid, out->loss,
                 out->q_num, out->q_den)) {
        out->valid = 1;
        out->bin = b;
        out->loss = loss;
        out->q_num = num;
        out->q_den = den;
        out->n_left = (double)nl;
        out->n_right = (double)nr;
      }
    } else {
      /* n * H_w = (n_L ln n_L - sum_k n_Lk ln n_Lk)
       *         + (n_R ln n_R - sum_k n_Rk ln n_Rk)  (natural log). */
      double sl = 0.0, sr = 0.0;
      for (int k = 0; k < K; ++k) sl += xlogx((double)left[k]);
      for (int k = 0; k < K; ++k) sr += xlogx((double)(tot[k] - left[k]));
      double h = (xlogx((double)nl) - sl) + (xlogx((double)nr) - sr);
      double loss = h / (double)ntot;
      if (out->valid && near_tie(loss, out->loss)) *tie = 1;
      if (!out->valid || loss < out->loss) {
        out->valid = 1;
        out->bin = b;
        out->loss = loss;
        out->n_left = (double)nl;
        out->n_right = (double)nr;
      }
    }
  }
}

/* Scores one projection vector a (as double; float-valued in the float
 * modes) with projection arithmetic `proj`. scratch: n_idx doubles for z,
 * n_idx doubles for the error bounds of PROJ_BF16, n_idx ints for bins, hist
 * buffers. *tie: a near-tie of double losses; *event: (PROJ_BF16) a sample
 * whose dot product another exact-product, float-accumulating evaluation
 * could round differently lies close enough to a bin edge to change bins. */
static void eval_one(const ora_params* p, int proj, const float* X, int32_t d,
                     const int32_t* labels, const float* y, const int32_t* idx,
                     const uint32_t* wts, int64_t n_idx, const double* a,
                     ora_eval* out, double* z, double* zb, int32_t* bins,
                     uint64_t* cnt, double* msum, double* msq, int* tie,
                     int* event) {
  const int B = p->n_bins;
  memset(out, 0, sizeof(*out));
  out->valid = 0;
  out->bin = -1;
  out->loss = INFINITY;

  /* Eq. (1): z = a^T x for every sample of the node. */
  double bmax = 0.0;
  for (int64_t s = 0; s < n_idx; ++s) {
    const float* xs = X + (int64_t)idx[s] * d;
    if (proj == PROJ_F32) {
      float acc = 0.0f;
      for (int32_t j = 0; j < d; ++j) acc = fmaf(xs[j], (float)a[j], acc);
      z[s] = acc;
    } else if (proj == PROJ_BF16) {
      /* bfloat16 products are exact in double; their sum is formed in double
       * and rounded once to float. Exact when every term is a multiple of
       * 2^L and sum |terms| < 2^(L+24): then every partial sum is a float. */
      double acc = 0.0, sabs = 0.0;
      int L = 1 << 20;
      for (int32_t j = 0; j < d; ++j) {
        double t = (double)bf16_round(xs[j]) * (double)bf16_round((float)a[j]);
        acc += t;
        sabs += fabs(t);
        if (t != 0.0) {
          int l = lsb_exponent(t);
          if (l < L) L = l;
        }
      }
      z[s] = (double)(float)acc;
      double bound = 0.0;
      if (sabs > 0.0 && !(sabs < ldexp(1.0, L + 24)))
        bound = (double)((d + 15) / 16 + 1) * ldexp(sabs, -22);
      zb[s] = bound;
      if (bound > bmax) bmax = bound;
    } else {
      double acc = 0.0;
      for (int32_t j = 0; j < d; ++j) acc += (double)xs[j] * a[j];
      z[s] = acc;
    }
  }
  if (n_idx <= 0) return;
  double zmin = z[0], zmax = z[0];
  for (int64_t s = 1; s < n_idx; ++s) {
    if (z[s] < zmin) zmin = z[s];
    if (z[s] > zmax) zmax = z[s];
  }
  out->zmin = zmin;
  out->zmax = zmax;
  if (!(zmax > zmin)) {
    if (proj == PROJ_BF16 && bmax > 0.0) *event = 1;
    return; /* every sample projects to one point */
  }

  /* Uniform bins on [zmin, zmax]: bin = min(B-1, floor((z-zmin)*inv_w)). */
  if (proj != PROJ_F64) {
    float fzmin = (float)zmin, fzmax = (float)zmax;
    float width = fzmax - fzmin;
    float inv_w = (float)B / width;
    if (!isfinite(inv_w)) return;
    out->inv_w = inv_w;
    for (int64_t s = 0; s < n_idx; ++s) {
      float off = (float)z[s] - fzmin;
      float pos = off * inv_w;
      int b = (int)floorf(pos);
      if (b > B - 1) b = B - 1;
      if (b < 0) b = 0;
      bins[s] = b;
      if (proj == PROJ_BF16 && bmax > 0.0) {
        /* edges move with zmin / zmax by at most bmax each */
        double margin = (zb[s] + 2.0 * bmax) * (double)inv_w + ldexp((double)B, -21);
        double k = floor((double)pos + 0.5);
        if (k >= 1.0 && k <= (double)(B - 1) && fabs((double)pos - k) <= margin) *event = 1;
      }
    }
  } else {
    double inv_w = (double)B / (zmax - zmin);
    if (!isfinite(inv_w)) return;
    out->inv_w = inv_w;
    for (int64_t s = 0; s < n_idx; ++s) {
      int b = (int)floor((z[s] - zmin) * inv_w);
      if (b > B - 1) b = B - 1;
      if (b < 0) b = 0;
      bins[s] = b;
    }
  }
  double keep_zmin = out->zmin, keep_zmax = out->zmax, keep_inv = out->inv_w;
  score_bins_into(p, labels, y, idx, wts, n_idx, bins, out, cnt, msum, msq, tie);
  out->zmin = keep_zmin;
  out->zmax = keep_zmax;
  out->inv_w = keep_inv;
}

static int check_params(const ora_params* p, int32_t d) {
  if (!p || d <= 0 || p->n_bins < 2 || p->min_leaf < 1) return -1;
  if (p->criterion == ORA_MSE) return 0;
  if (p->criterion != ORA_GINI && p->criterion != ORA_ENTROPY) return -1;
  if (p->n_classes < 2 || p->n_classes > 64) return -1;
  return 0;
}

/* Scores particles sel[0..m) (sel NULL: 0..m-1) of pos[*, d]; out[q] is
 * the score of particle sel[q]. */
static int eval_all(const ora_params* p, int proj, const float* X, int32_t d,
                    const int32_t* labels, const float* y, const int32_t* idx,
                    const uint32_t* wts, int64_t n_idx, const double* pos,
                    const int32_t* sel, int32_t m, ora_eval* out,
                    int32_t* bins_out, double* z_out, int* tie_any,
                    int* event_any) {
  const int B = p->n_bins;
  const int K = p->criterion == ORA_MSE ? 1 : p->n_classes;
  int err = 0;
  int tie = 0, event = 0;
#ifdef _OPENMP
  int nt = p->n_threads > 0 ? p->n_threads : omp_get_max_threads();
#pragma omp parallel num_threads(nt) reduction(| : err, tie, event)
#endif
  {
    size_t nz = (size_t)(n_idx > 0 ? n_idx : 1);
    double* z = (double*)malloc(sizeof(double) * nz);
    double* zb = (double*)malloc(sizeof(double) * nz);
    int32_t* bins = (int32_t*)malloc(sizeof(int32_t) * nz);
    uint64_t* cnt = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)B * K);
    double* msum = (double*)malloc(sizeof(double) * (size_t)B);
    double* msq = (double*)malloc(sizeof(double) * (size_t)B);
    if (!z || !zb || !bins || !cnt || !msum || !msq) {
      err = 1;
    } else {
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
      for (int32_t q = 0; q < m; ++q) {
        const int32_t i = sel ? sel[q] : q;
        int t = 0, ev = 0;
        for (int64_t s = 0; s < n_idx; ++s) bins[s] = -1;
        eval_one(p, proj, X, d, labels, y, idx, wts, n_idx, pos + (int64_t)i * d,
                 &out[q], z, zb, bins, cnt, msum, msq, &t, &ev);
        tie |= t;
        event |= ev;
        if (bins_out)
          memcpy(bins_out + (int64_t)q * n_idx, bins, sizeof(int32_t) * (size_t)n_idx);
        if (z_out) memcpy(z_out + (int64_t)q * n_idx, z, sizeof(double) * (size_t)n_idx);
      }
    }
    free(z);
    free(zb);
    free(bins);
    free(cnt);
    free(msum);
    free(msq);
  }
  if (tie_any) *tie_any = tie;
  if (event_any) *event_any = event;
  return err ? -2 : 0;
}

static int proj_of(const ora_params* p) {
  return p->precision == ORA_F64 ? PROJ_F64
                                 : p->precision == ORA_F32_MIRROR ? PROJ_F32 : PROJ_BF16;
}

/* The k particles with the best scores ev[0..P), ties to the lower index,
 * returned in increasing particle order. *tie: the k-th and the (k+1)-th
 * best are a near-tie of double losses. */
static void select_topk(const ora_params* p, const ora_eval* ev, int32_t P,
                        int32_t k, int32_t* sel, int* tie) {
  char* taken = (char*)calloc((size_t)P, 1);
  int32_t last = -1;
  for (int32_t q = 0; q <= k && q < P; ++q) {
    int32_t best = -1;
    for (int32_t i = 0; i < P; ++i) {
      if (taken[i]) continue;
      if (best < 0 || better(p->criterion, ev[i].valid, ev[i].loss, ev[i].q_num,
                             ev[i].q_den, ev[best].valid, ev[best].loss,
                             ev[best].q_num, ev[best].q_den))
        best = i;
    }
    if (q == k) { /* first one left out */
      if (p->criterion != ORA_GINI && last >= 0 && ev[best].valid && ev[last].valid &&
          near_tie(ev[best].loss, ev[last].loss))
        *tie = 1;
      break;
    }
    taken[best] = 1;
    last = best;
  }
  int32_t c = 0;
  for (int32_t i = 0; i < P && c < k; ++i)
    if (taken[i]) sel[c++] = i;
  free(taken);
}

int ora_eval_swarm(const ora_params* p, const float* X, int32_t d,
                   const int32_t* labels, const float* y, const int32_t* idx,
                   const uint32_t* wts, int64_t n_idx, const double* pos,
                   int32_t P, ora_eval* out, int32_t* bins_out,
                   double* z_out) {
  if (check_params(p, d) || P < 1 || n_idx < 0 || !X || !idx || !pos || !out)
    return -1;
  int rc = eval_all(p, proj_of(p), X, d, labels, y, idx, wts, n_idx, pos, NULL, P,
                    out, bins_out, z_out, NULL, NULL);
  if (rc || p->precision != ORA_BF16_TOPK || p->topk <= 0) return rc;
  const int32_t k = p->topk < P ? p->topk : P;
  int32_t* sel = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  ora_eval* ef = (ora_eval*)malloc(sizeof(ora_eval) * (size_t)k);
  if (!sel || !ef) {
    free(sel);
    free(ef);
    return -2;
  }
  int tie = 0;
  select_topk(p, out, P, k, sel, &tie);
  rc = eval_all(p, PROJ_F32, X, d, labels, y, idx, wts, n_idx, pos, sel, k, ef,
                NULL, NULL, NULL, NULL);
  for (int32_t q = 0; q < k && !rc; ++q) out[sel[q]] = ef[q];
  free(sel);
  free(ef);
  return rc;
}

int ora_score_bins(const ora_params* p, const int32_t* labels, const float* y,
                   const int32_t* idx, const uint32_t* wts, int64_t n_idx,
                   const int32_t* bins, ora_eval* out) {
  if (check_params(p, 1) || n_idx < 0 || !idx || !bins || !out) return -1;
  if (p->criterion == ORA_MSE ? !y : !labels) return -1;
  for (int64_t s = 0; s < n_idx; ++s)
    if (bins[s] < 0 || bins[s] >= p->n_bins) return -1;
  const int B = p->n_bins;
  const int K = p->criterion == ORA_MSE ? 1 : p->n_classes;
  uint64_t* cnt = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)B * K);
  double* msum = (double*)malloc(sizeof(double) * (size_t)B);
  double* msq = (double*)malloc(sizeof(double) * (size_t)B);
  int rc = 0;
  if (!cnt || !msum || !msq) {
    rc = -2;
  } else {
    int tie = 0;
    memset(out, 0, sizeof(*out));
    score_bins_into(p, labels, y, idx, wts, n_idx, bins, out, cnt, msum, msq, &tie);
  }
  free(cnt);
  free(msum);
  free(msq);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Elitist learning of the adaptive PSO (Sec. III-B; the cited APSO method's  */
/* rule for the convergence state): a copy of gB with one coordinate moved   */
/* by a Gaussian step is scored; it becomes gB if better, otherwise it takes */
/* the place of the worst particle.                                          */

void ora_elite_candidate(uint64_t seed, uint32_t node_uid, uint32_t t, int32_t T, int32_t d,
                         const double* gb, int32_t precision, double* e, int32_t* k_out) {
  float u[4];
  ora_swarm_uniforms(seed, node_uid, t, 1, 4, ORA_PURPOSE_APSO, u);
  const int32_t k = (int32_t)((double)u[1] * (double)d);
  const double g = sqrt(-2.0 * log((double)(1.0f - u[2]))) *
                   cos(6.283185307179586 * (double)u[3]);
  for (int32_t j = 0; j < d; ++j) e[j] = gb[j];
  if (precision == ORA_F64) {
    const double sigma = 1.0 - 0.9 * ((double)t / (double)T);
    e[k] = gb[k] + 2.0 * sigma * g;
  } else {
    const float sigma = 1.0f - 0.9f * ((float)t / (float)T);
    e[k] = (double)((float)gb[k] + (2.0f * sigma) * (float)g);
  }
  if (k_out) *k_out = k;
}

#define EV_ARGS(e) (e)->valid, (e)->loss, (e)->q_num, (e)->q_den

/* The acceptance step on scored positions: ev / pbe the particles' current
 * and personal-best scores, gbe gB's score; returns 1 when the candidate
 * (score ee, position elite) became gB, else 0 with the replaced particle in
 * *worst. Near-ties of the comparisons that decide are flagged in *tie. */
static int elite_apply(int crit, int32_t P, int32_t d, double* x, double* pb, ora_eval* ev,
                       ora_eval* pbe, ora_eval* gbe, int32_t gpart, double* gb,
                       const double* elite, const ora_eval* ee, int* tie, int32_t* worst) {
  if (gbe->valid && ee->valid && near_tie(ee->loss, gbe->loss)) *tie = 1;
  if (better(crit, EV_ARGS(ee), EV_ARGS(gbe))) {
    *gbe = *ee;
    pbe[gpart] = *ee;
    memcpy(gb, elite, sizeof(double) * d);
    memcpy(pb + (int64_t)gpart * d, elite, sizeof(double) * d);
    return 1;
  }
  int32_t w = 0;
  for (int32_t i = 1; i < P; ++i)
    if (better(crit, EV_ARGS(&ev[w]), EV_ARGS(&ev[i]))) w = i; /* i strictly worse */
  for (int32_t i = 0; i < P; ++i)
    if (i != w && ev[i].valid && ev[w].valid && near_tie(ev[i].loss, ev[w].loss)) *tie = 1;
  memcpy(x + (int64_t)w * d, elite, sizeof(double) * d);
  ev[w] = *ee;
  if (pbe[w].valid && ee->valid && near_tie(ee->loss, pbe[w].loss)) *tie = 1;
  if (better(crit, EV_ARGS(ee), EV_ARGS(&pbe[w]))) {
    pbe[w] = *ee;
    memcpy(pb + (int64_t)w * d, elite, sizeof(double) * d);
  }
  *worst = w;
  return 0;
}

static ora_eval loss_eval(double loss) {
  ora_eval e;
  memset(&e, 0, sizeof(e));
  e.valid = isfinite(loss) ? 1 : 0;
  e.loss = loss;
  return e;
}

int32_t ora_elite_apply(int32_t P, int32_t d, double* x, double* pb, double* cur_loss,
                        double* pb_loss, double* g_loss, int32_t gpart, double* gb,
                        const double* elite, double e_loss, int32_t* worst_out) {
  if (P < 1 || d < 1 || gpart < 0 || gpart >= P) return -1;
  ora_eval* ev = (ora_eval*)calloc((size_t)P, sizeof(ora_eval));
  ora_eval* pbe = (ora_eval*)calloc((size_t)P, sizeof(ora_eval));
  if (!ev || !pbe) {
    free(ev);
    free(pbe);
    return -2;
  }
  for (int32_t i = 0; i < P; ++i) {
    ev[i] = loss_eval(cur_loss[i]);
    pbe[i] = loss_eval(pb_loss[i]);
  }
  ora_eval gbe = loss_eval(*g_loss), ee = loss_eval(e_loss);
  int tie = 0;
  int32_t w = -1;
  const int acc = elite_apply(ORA_MSE, P, d, x, pb, ev, pbe, &gbe, gpart, gb, elite, &ee, &tie,
                              &w);
  for (int32_t i = 0; i < P; ++i) {
    cur_loss[i] = ev[i].valid ? ev[i].loss : INFINITY;
    pb_loss[i] = pbe[i].valid ? pbe[i].loss : INFINITY;
  }
  *g_loss = gbe.valid ? gbe.loss : INFINITY;
  if (worst_out) *worst_out = w;
  free(ev);
  free(pbe);
  return acc;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (PSO), synchronous form: every particle moves with the gbest  */
/* held at the end of the previous iteration, then all are scored, then     */
/* pbest and gbest are updated with strict "<" in increasing particle order. */

static void copy_eval_to_split(const ora_eval* e, ora_split* s) {
  s->valid = e->valid;
  s->bin = e->bin;
  s->zmin = e->zmin;
  s->inv_w = e->inv_w;
  s->loss = e->loss;
  s->q_num = e->q_num;
  s->q_den = e->q_den;
  s->n_left = e->n_left;
  s->n_right = e->n_right;
}

static int node_split_full(const ora_params* p, const float* X, int32_t d,
                           const int32_t* labels, const float* y, const int32_t* idx,
                           const uint32_t* wts, int64_t n_idx, uint32_t node_uid,
                           const float* init_x, double* gbest_out, double* dir_out,
                           ora_split* out, double* trace_loss, int32_t* trace_particle) {
  if (check_params(p, d) || p->n_particles < 1 || p->n_iters < 0 || n_idx < 0 ||
      !X || !idx || !out || (p->precision == ORA_BF16_TOPK && p->topk < 1) ||
      (p->apso && p->precision == ORA_BF16_TOPK))
    return -1;
  const int32_t P = p->n_particles;
  const int32_t T = p->n_iters;
  const int64_t PD = (int64_t)P * d;
  double* x = (double*)calloc((size_t)PD, sizeof(double));
  double* v = (double*)calloc((size_t)PD, sizeof(double));
  double* pb = (double*)calloc((size_t)PD, sizeof(double));
  double* gb = (double*)calloc((size_t)d, sizeof(double));
  double* r1 = (double*)calloc((size_t)PD, sizeof(double));
  double* r2 = (double*)calloc((size_t)PD, sizeof(double));
  float* u = (float*)calloc((size_t)PD, sizeof(float));
  ora_eval* ev = (ora_eval*)calloc((size_t)P, sizeof(ora_eval));
  ora_eval* pbe = (ora_eval*)calloc((size_t)P, sizeof(ora_eval));
  const int bf16 = p->precision == ORA_BF16_TOPK;
  const int32_t k = bf16 ? (p->topk < P ? p->topk : P) : 0;
  int32_t* sel = (int32_t*)calloc((size_t)(k > 0 ? k : 1), sizeof(int32_t));
  ora_eval* ef = (ora_eval*)calloc((size_t)(k > 0 ? k : 1), sizeof(ora_eval));
  double* elite = (double*)calloc((size_t)d, sizeof(double));
  int rc = 0;
  if (!x || !v || !pb || !gb || !r1 || !r2 || !u || !ev || !pbe || !sel || !ef || !elite) {
    rc = -2;
    goto done;
  }
  memset(out, 0, sizeof(*out));
  out->first_near_tie = -1;

  /* Initial swarm: x ~ U[-1,1)^d (or the given start, e.g. a learned seed),
   * v ~ 0.1 * U[-1,1)^d. */
  ora_swarm_uniforms(p->seed, node_uid, 0, P, d, ORA_PURPOSE_INIT_X, u);
  for (int64_t e = 0; e < PD; ++e) x[e] = init_x ? (double)init_x[e] : (double)(2.0f * u[e] - 1.0f);
  ora_swarm_uniforms(p->seed, node_uid, 0, P, d, ORA_PURPOSE_INIT_V, u);
  for (int64_t e = 0; e < PD; ++e) {
    if (p->precision != ORA_F64)
      v[e] = (double)(0.1f * (2.0f * u[e] - 1.0f));
    else
      v[e] = 0.1 * (double)(2.0f * u[e] - 1.0f);
  }

  ora_eval gbe;
  memset(&gbe, 0, sizeof(gbe));
  int32_t gpart = 0, giter = 0;
  ora_params q = *p;  /* the move's inertia and learning factors */
  int32_t astate = ORA_APSO_EXPLORE;
  int pending = 0; /* an elite candidate waits for this evaluation */
  for (int32_t t = 0; t <= T; ++t) {
    if (t > 0) {
      ora_swarm_uniforms(p->seed, node_uid, (uint32_t)t, P, d, ORA_PURPOSE_R1, u);
      for (int64_t e = 0; e < PD; ++e) r1[e] = u[e];
      ora_swarm_uniforms(p->seed, node_uid, (uint32_t)t, P, d, ORA_PURPOSE_R2, u);
      for (int64_t e = 0; e < PD; ++e) r2[e] = u[e];
      ora_pso_step(&q, P, d, x, v, pb, gb, r1, r2);
    }
    int tie = 0, event = 0;
    rc = eval_all(p, proj_of(p), X, d, labels, y, idx, wts, n_idx, x, NULL, P, ev,
                  NULL, NULL, &tie, &event);
    if (rc) goto done;
    if (bf16) {
      /* re-score the k best on the float projection; their scores replace
       * the bfloat16 ones */
      int tie2 = 0;
      select_topk(p, ev, P, k, sel, &tie);
      rc = eval_all(p, PROJ_F32, X, d, labels, y, idx, wts, n_idx, x, sel, k, ef,
                    NULL, NULL, &tie2, NULL);
      if (rc) goto done;
      tie |= tie2;
      for (int32_t q = 0; q < k; ++q) ev[sel[q]] = ef[q];
    }
    for (int32_t i = 0; i < P; ++i) {
      const ora_eval* e = &ev[i];
      int improved = 0;
      if (t == 0) {
        improved = 1; /* pbest starts at the initial position */
      } else {
        if (pbe[i].valid && e->valid && near_tie(e->loss, pbe[i].loss)) tie = 1;
        improved = better(p->criterion, e->valid, e->loss, e->q_num, e->q_den,
                          pbe[i].valid, pbe[i].loss, pbe[i].q_num, pbe[i].q_den);
      }
      if (!improved) continue;
      pbe[i] = *e;
      memcpy(pb + (int64_t)i * d, x + (int64_t)i * d, sizeof(double) * d);
      if (bf16) continue; /* gbest below, from the re-scored particles */
      int first = (t == 0 && i == 0);
      if (!first && gbe.valid && e->valid && near_tie(e->loss, gbe.loss)) tie = 1;
      if (first || better(p->criterion, e->valid, e->loss, e->q_num, e->q_den,
                          gbe.valid, gbe.loss, gbe.q_num, gbe.q_den)) {
        gbe = *e;
        gpart = i;
        giter = t;
        memcpy(gb, x + (int64_t)i * d, sizeof(double) * d);
      }
    }
    for (int32_t q = 0; bf16 && q < k; ++q) {
      const int32_t i = sel[q];
      const ora_eval* e = &ev[i];
      int first = (t == 0 && q == 0);
      if (!first && gbe.valid && e->valid && near_tie(e->loss, gbe.loss)) tie = 1;
      if (first || better(p->criterion, e->valid, e->loss, e->q_num, e->q_den,
                          gbe.valid, gbe.loss, gbe.q_num, gbe.q_den)) {
        gbe = *e;
        gpart = i;
        giter = t;
        memcpy(gb, x + (int64_t)i * d, sizeof(double) * d);
      }
    }
    if (pending) {
      /* the elite candidate made after evaluation t-1, scored with this
       * evaluation, after the particles' pbest and gbest steps */
      ora_eval ee;
      int tie_e = 0, event_e = 0;
      int32_t w;
      rc = eval_all(p, proj_of(p), X, d, labels, y, idx, wts, n_idx, elite, NULL, 1, &ee, NULL,
                    NULL, &tie_e, &event_e);
      if (rc) goto done;
      tie |= tie_e;
      event |= event_e;
      ++out->elite_tries;
      if (elite_apply(p->criterion, P, d, x, pb, ev, pbe, &gbe, gpart, gb, elite, &ee, &tie,
                      &w)) {
        giter = t;
        ++out->elite_accepts;
      }
      pending = 0;
    }
    if (p->criterion == ORA_GINI) tie = 0; /* exact rationals: no near-ties */
    if ((tie || event) && out->first_near_tie < 0) out->first_near_tie = t;
    if (trace_loss) trace_loss[t] = gbe.valid ? gbe.loss : INFINITY;
    if (trace_particle) trace_particle[t] = gpart;
    if (p->apso && t < T) {
      /* the state after evaluation t sets the move to iteration t + 1 */
      float du;
      ora_swarm_uniforms(p->seed, node_uid, (uint32_t)t, 1, 1, ORA_PURPOSE_APSO, &du);
      ora_apso st;
      ora_apso_step(P, d, x, gpart, astate, q.c1, q.c2, 0.05f + 0.05f * du, &st);
      astate = st.state;
      q.c1 = st.c1;
      q.c2 = st.c2;
      q.inertia = st.w;
      if (astate == ORA_APSO_CONVERGE) {
        ora_elite_candidate(p->seed, node_uid, (uint32_t)t, T, d, gb, p->precision, elite,
                            NULL);
        pending = 1;
      }
    }
  }

  copy_eval_to_split(&gbe, out);
  out->particle = gpart;
  out->iter_of_best = giter;
  if (gbe.valid) {
    if (p->precision != ORA_F64)
      out->threshold = (double)((float)gbe.zmin + (float)gbe.bin / (float)gbe.inv_w);
    else
      out->threshold = gbe.zmin + (double)gbe.bin / gbe.inv_w;
  }
  if (gbest_out) memcpy(gbest_out, gb, sizeof(double) * d);
  if (dir_out) {
    double nrm = 0.0;
    for (int32_t j = 0; j < d; ++j) nrm += gb[j] * gb[j];
    nrm = sqrt(nrm);
    for (int32_t j = 0; j < d; ++j) dir_out[j] = nrm > 0.0 ? gb[j] / nrm : 0.0;
  }

done:
  free(x);
  free(v);
  free(pb);
  free(gb);
  free(r1);
  free(r2);
  free(u);
  free(ev);
  free(pbe);
  free(sel);
  free(ef);
  free(elite);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: grow a binary tree breadth-first.                           */

typedef struct {
  int32_t* idx;
  uint32_t* w;
  int64_t n;
} node_samples;

/* Bin of sample x under a stored split, in the mode's precision. */
static int split_bin(const ora_params* p, const double* dir, double zmin,
                     double inv_w, const float* xs, int32_t d) {
  const int B = p->n_bins;
  int b;
  if (p->precision != ORA_F64) {
    float acc = 0.0f;
    for (int32_t j = 0; j < d; ++j) acc = fmaf(xs[j], (float)dir[j], acc);
    float off = acc - (float)zmin;
    float pos = off * (float)inv_w;
    b = (int)floorf(pos);
  } else {
    double acc = 0.0;
    for (int32_t j = 0; j < d; ++j) acc += (double)xs[j] * dir[j];
    b = (int)floor((acc - zmin) * inv_w);
  }
  if (b > B - 1) b = B - 1;
  if (b < 0) b = 0;
  return b;
}


/* Per-node feature pre-screen (Sec. III-B, Algorithm 2): the split loss of
 * every feature on its own (the projection on the unit vector e_k, scored
 * like any particle; z = x_k exactly), the n = top_n best kept (ties to the
 * lower feature, increasing feature order: select_topk's rule). */
int ora_select_features(const ora_params* p, const float* X, int32_t d,
                        const int32_t* labels, const float* y, const int32_t* idx,
                        const uint32_t* wts, int64_t n_idx, int32_t n, int32_t* feat,
                        ora_eval* ev_out, int32_t* near_tie) {
  if (check_params(p, d) || n < 1 || n > d || !feat) return -1;
  double* eye = (double*)calloc((size_t)d * d, sizeof(double));
  ora_eval* ev = (ora_eval*)calloc((size_t)d, sizeof(ora_eval));
  int rc = 0;
  if (!eye || !ev) {
    rc = -2;
    goto done;
  }
  for (int32_t k = 0; k < d; ++k) eye[(int64_t)k * d + k] = 1.0;
  int tie = 0, event = 0;
  rc = eval_all(p, p->precision == ORA_F64 ? PROJ_F64 : PROJ_F32, X, d, labels, y, idx, wts,
                n_idx, eye, NULL, d, ev, NULL, NULL, &tie, &event);
  if (rc) goto done;
  int sel_tie = 0;
  select_topk(p, ev, d, n, feat, &sel_tie);
  if (near_tie) *near_tie = sel_tie;
  if (ev_out) memcpy(ev_out, ev, sizeof(ora_eval) * (size_t)d);
done:
  free(eye);
  free(ev);
  return rc;
}

int ora_node_split(const ora_params* p, const float* X, int32_t d,
                   const int32_t* labels, const float* y, const int32_t* idx,
                   const uint32_t* wts, int64_t n_idx, uint32_t node_uid,
                   double* gbest_out, double* dir_out, ora_split* out,
                   double* trace_loss, int32_t* trace_particle) {
  const int32_t n = p ? p->top_n : 0;
  if (n <= 0 || n >= d)
    return node_split_full(p, X, d, labels, y, idx, wts, n_idx, node_uid, NULL, gbest_out,
                           dir_out, out, trace_loss, trace_particle);
  /* the swarm searches the n-dimensional subspace of the selected features;
   * its direction is lifted back with zeros elsewhere */
  if (check_params(p, d) || !X || !idx || n_idx < 0 || !out) return -1;
  int32_t* feat = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  int64_t rows = 0;
  for (int64_t i = 0; i < n_idx; ++i)
    if ((int64_t)idx[i] + 1 > rows) rows = (int64_t)idx[i] + 1;
  float* Xs = (float*)calloc((size_t)(rows > 0 ? rows : 1) * n, sizeof(float));
  double* gs = (double*)calloc((size_t)n, sizeof(double));
  double* ds = (double*)calloc((size_t)n, sizeof(double));
  int rc = 0, tie = 0;
  if (!feat || !Xs || !gs || !ds) {
    rc = -2;
    goto done;
  }
  rc = ora_select_features(p, X, d, labels, y, idx, wts, n_idx, n, feat, NULL, &tie);
  if (rc) goto done;
  for (int64_t i = 0; i < n_idx; ++i) {
    const int64_t r = idx[i];
    for (int32_t j = 0; j < n; ++j) Xs[r * n + j] = X[r * d + feat[j]];
  }
  rc = node_split_full(p, Xs, n, labels, y, idx, wts, n_idx, node_uid, NULL, gs, ds, out,
                       trace_loss, trace_particle);
  if (rc) goto done;
  if (gbest_out)
    for (int32_t k = 0; k < d; ++k) gbest_out[k] = 0.0;
  if (dir_out)
    for (int32_t k = 0; k < d; ++k) dir_out[k] = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    if (gbest_out) gbest_out[feat[j]] = gs[j];
    if (dir_out) dir_out[feat[j]] = ds[j];
  }
  if (tie) out->first_near_tie = 0;  /* another selection is as correct */
done:
  free(feat);
  free(Xs);
  free(gs);
  free(ds);
  return rc;
}

int ora_node_split_from(const ora_params* p, const float* X, int32_t d,
                        const int32_t* labels, const float* y, const int32_t* idx,
                        const uint32_t* wts, int64_t n_idx, uint32_t node_uid,
                        const float* init_x, double* gbest_out, double* dir_out,
                        ora_split* out, double* trace_loss, int32_t* trace_particle) {
  if (!init_x || (p && p->top_n > 0 && p->top_n < d)) return -1;
  return node_split_full(p, X, d, labels, y, idx, wts, n_idx, node_uid, init_x, gbest_out,
                         dir_out, out, trace_loss, trace_particle);
}

/* ------------------------------------------------------------------------ */
/* Probabilistic search (Sec. II-B).                                        */

void ora_prob_candidate(uint64_t seed, uint32_t node_uid, uint32_t c, int32_t d,
                        const int32_t* rank_feat, const ora_prob* pp, double* a_out) {
  uint32_t key[2];
  seed_key(seed, key);
  const int32_t R = pp->R < d ? pp->R : d;
  double* w = (double*)malloc(sizeof(double) * (size_t)d);
  char* used = (char*)calloc((size_t)d, 1);
  int32_t* chosen = (int32_t*)malloc(sizeof(int32_t) * (size_t)(R > 0 ? R : 1));
  for (int32_t j = 0; j < d; ++j) a_out[j] = 0.0;
  if (!w || !used || !chosen) goto done;
  w[0] = 1.0;
  for (int32_t r = 1; r < d; ++r) w[r] = w[r - 1] * pp->gamma;  /* P_r, rank r + 1 */
  for (int32_t k = 0; k < 2 * R; ++k) {
    uint32_t ctr[4] = {node_uid, c, (uint32_t)k >> 2, (uint32_t)ORA_PURPOSE_PROB << 24};
    uint32_t rr[4];
    ora_philox4x32_10(ctr, key, rr);
    const double u = (double)u01(rr[k & 3]);
    if (k < R) {
      double total = 0.0;
      for (int32_t r = 0; r < d; ++r)
        if (!used[r]) total += w[r];
      const double target = u * total;
      double run = 0.0;
      int32_t pick = -1, last = -1;
      for (int32_t r = 0; r < d; ++r) {
        if (used[r]) continue;
        last = r;
        run += w[r];
        if (run > target) {
          pick = r;
          break;
        }
      }
      if (pick < 0) pick = last;
      used[pick] = 1;
      chosen[k] = pick;
    } else {
      const int32_t r = chosen[k - R];  /* 0-based rank: A of rank r + 1 */
      const double m = floor(pp->alpha0 * exp(-pp->alpha * (double)(r + 1)));
      a_out[rank_feat[r]] = floor(u * (2.0 * m + 1.0)) - m;
    }
  }
done:
  free(w);
  free(used);
  free(chosen);
}

int ora_prob_search(const ora_params* p, const ora_prob* pp, const float* X, int32_t d,
                    const int32_t* labels, const float* y, const int32_t* idx,
                    const uint32_t* wts, int64_t n_idx, uint32_t node_uid, double* best_out,
                    ora_split* out, double* trace_loss, int32_t* rank_feat_out, int32_t* kept,
                    int32_t* n_kept) {
  if (check_params(p, d) || !pp || pp->n_candidates < 1 || pp->R < 1 || pp->batch < 1 ||
      !(pp->gamma > 0.0 && pp->gamma <= 1.0) || pp->q < 0 || pp->cos_den < 1 ||
      pp->cos_num < 0 || !X || !idx || n_idx < 0 || !out || p->precision == ORA_BF16_TOPK)
    return -1;
  const int32_t I = pp->n_candidates;
  double* eye = (double*)calloc((size_t)d * d, sizeof(double));
  ora_eval* fe = (ora_eval*)calloc((size_t)d, sizeof(ora_eval));
  int32_t* rank_feat = (int32_t*)malloc(sizeof(int32_t) * (size_t)d);
  char* taken = (char*)calloc((size_t)d, 1);
  double* cand = (double*)malloc(sizeof(double) * (size_t)I * d);
  ora_eval* ev = (ora_eval*)calloc((size_t)I, sizeof(ora_eval));
  char* pruned = (char*)calloc((size_t)I, 1);
  int rc = 0;
  if (!eye || !fe || !rank_feat || !taken || !cand || !ev || !pruned) {
    rc = -2;
    goto done;
  }
  memset(out, 0, sizeof(*out));
  out->first_near_tie = -1;
  /* rank the features by their own split loss, better first */
  for (int32_t k = 0; k < d; ++k) eye[(int64_t)k * d + k] = 1.0;
  rc = eval_all(p, proj_of(p), X, d, labels, y, idx, wts, n_idx, eye, NULL, d, fe, NULL, NULL,
                NULL, NULL);
  if (rc) goto done;
  for (int32_t r = 0; r < d; ++r) {
    int32_t best = -1;
    for (int32_t k = 0; k < d; ++k) {
      if (taken[k]) continue;
      if (best < 0 || better(p->criterion, fe[k].valid, fe[k].loss, fe[k].q_num, fe[k].q_den,
                             fe[best].valid, fe[best].loss, fe[best].q_num, fe[best].q_den))
        best = k;
    }
    taken[best] = 1;
    rank_feat[r] = best;
  }
  if (rank_feat_out) memcpy(rank_feat_out, rank_feat, sizeof(int32_t) * (size_t)d);
  /* generate and score the candidates; the best so far after each batch */
  for (int32_t c = 0; c < I; ++c)
    ora_prob_candidate(p->seed, node_uid, (uint32_t)c, d, rank_feat, pp, cand + (int64_t)c * d);
  rc = eval_all(p, proj_of(p), X, d, labels, y, idx, wts, n_idx, cand, NULL, I, ev, NULL, NULL,
                NULL, NULL);
  if (rc) goto done;
  int32_t bi = 0;
  for (int32_t c = 0; c < I; ++c) {
    if (c > 0 && better(p->criterion, ev[c].valid, ev[c].loss, ev[c].q_num, ev[c].q_den,
                        ev[bi].valid, ev[bi].loss, ev[bi].q_num, ev[bi].q_den))
      bi = c;
    if (trace_loss && ((c + 1) % pp->batch == 0 || c == I - 1))
      trace_loss[c / pp->batch] = ev[bi].valid ? ev[bi].loss : INFINITY;
  }
  copy_eval_to_split(&ev[bi], out);
  out->particle = bi;
  out->iter_of_best = bi / pp->batch;
  if (ev[bi].valid) {
    if (p->precision != ORA_F64)
      out->threshold = (double)((float)ev[bi].zmin + (float)ev[bi].bin / (float)ev[bi].inv_w);
    else
      out->threshold = ev[bi].zmin + (double)ev[bi].bin / ev[bi].inv_w;
  }
  if (best_out) memcpy(best_out, cand + (int64_t)bi * d, sizeof(double) * d);
  /* cosine pruning: the best remaining, then drop its close neighbours */
  int32_t nk = 0;
  const int64_t cn2 = (int64_t)pp->cos_num * pp->cos_num, cd2 = (int64_t)pp->cos_den * pp->cos_den;
  while (nk < pp->q) {
    int32_t b = -1;
    for (int32_t c = 0; c < I; ++c) {
      if (pruned[c]) continue;
      int64_t nrm = 0;
      for (int32_t j = 0; j < d; ++j) nrm += (int64_t)cand[(int64_t)c * d + j] * (int64_t)cand[(int64_t)c * d + j];
      if (nrm == 0) {
        pruned[c] = 1;
        continue;
      }
      if (b < 0 || better(p->criterion, ev[c].valid, ev[c].loss, ev[c].q_num, ev[c].q_den,
                          ev[b].valid, ev[b].loss, ev[b].q_num, ev[b].q_den))
        b = c;
    }
    if (b < 0) break;
    if (kept) kept[nk] = b;
    ++nk;
    const double* ab = cand + (int64_t)b * d;
    int64_t na = 0;
    for (int32_t j = 0; j < d; ++j) na += (int64_t)ab[j] * (int64_t)ab[j];
    for (int32_t c = 0; c < I; ++c) {
      if (pruned[c]) continue;
      const double* ac = cand + (int64_t)c * d;
      int64_t dot = 0, nc = 0;
      for (int32_t j = 0; j < d; ++j) {
        dot += (int64_t)ab[j] * (int64_t)ac[j];
        nc += (int64_t)ac[j] * (int64_t)ac[j];
      }
      if (c == b || cd2 * dot * dot > cn2 * na * nc) pruned[c] = 1;
    }
  }
  if (n_kept) *n_kept = nk;
done:
  free(eye);
  free(fe);
  free(rank_feat);
  free(taken);
  free(cand);
  free(ev);
  free(pruned);
  return rc;
}

int ora_train_tree(const ora_params* p, const float* X, int64_t n, int32_t d,
                   const int32_t* labels, const float* y, uint32_t tree_id,
                   int32_t bootstrap, ora_tree* out) {
  if (check_params(p, d) || n < 1 || !X || !out || p->max_depth < 0 ||
      p->max_depth > 15)
    return -1;
  if (p->criterion == ORA_MSE ? !y : !labels) return -1;
  const int D = p->max_depth;
  const int64_t H = ((int64_t)1 << (D + 1)) - 1;
  const int K = p->n_classes;
  for (int64_t h = 0; h < H; ++h) {
    out->kind[h] = -1;
    out->zmin[h] = out->inv_w[h] = 0.0;
    out->bin[h] = -1;
    out->leaf_class[h] = -1;
    out->leaf_value[h] = 0.0;
    out->weight[h] = 0.0;
    out->loss[h] = 0.0;
    out->n_left[h] = out->n_right[h] = 0.0;
    for (int32_t j = 0; j < d; ++j) out->dir[h * d + j] = 0.0;
  }
  node_samples* ns = (node_samples*)calloc((size_t)H, sizeof(node_samples));
  if (!ns) return -2;
  int rc = 0;

  /* Root: every sample (weight 1), or the distinct bootstrap draws with
   * their multiplicities. */
  {
    uint32_t* bw = NULL;
    int64_t m = n;
    if (bootstrap) {
      bw = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
      if (!bw) { free(ns); return -2; }
      ora_bootstrap(p->seed, tree_id, n, bw);
      m = 0;
      for (int64_t s = 0; s < n; ++s) m += bw[s] > 0;
    }
    ns[0].idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    ns[0].w = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
    if (!ns[0].idx || !ns[0].w) { free(bw); rc = -2; goto done; }
    int64_t k = 0;
    for (int64_t s = 0; s < n; ++s) {
      uint32_t w = bw ? bw[s] : 1u;
      if (w == 0) continue;
      ns[0].idx[k] = (int32_t)s;
      ns[0].w[k] = w;
      ++k;
    }
    ns[0].n = k;
    free(bw);
  }

  double* gbest = (double*)malloc(sizeof(double) * d);
  uint64_t* cls = (uint64_t*)malloc(sizeof(uint64_t) * (K > 0 ? K : 1));
  if (!gbest || !cls) { free(gbest); free(cls); rc = -2; goto done; }

  for (int depth = 0; depth <= D && rc == 0; ++depth) {
    int64_t h0 = ((int64_t)1 << depth) - 1, h1 = ((int64_t)1 << (depth + 1)) - 1;
    for (int64_t h = h0; h < h1 && rc == 0; ++h) {
      if (!ns[h].idx) continue;
      node_samples* nd = &ns[h];
      /* Node statistics: weighted count, class counts or target moments. */
      uint64_t nw = 0;
      for (int64_t s = 0; s < nd->n; ++s) nw += nd->w[s];
      int pure = 0;
      if (p->criterion == ORA_MSE) {
        double sy = 0.0;
        float ymin = INFINITY, ymax = -INFINITY;
        for (int64_t s = 0; s < nd->n; ++s) {
          float ys = y[nd->idx[s]];
          sy += (double)nd->w[s] * (double)ys;
          if (ys < ymin) ymin = ys;
          if (ys > ymax) ymax = ys;
        }
        out->leaf_value[h] = nw ? sy / (double)nw : 0.0;
        pure = !(ymax > ymin);
      } else {
        for (int k = 0; k < K; ++k) cls[k] = 0;
        for (int64_t s = 0; s < nd->n; ++s) cls[labels[nd->idx[s]]] += nd->w[s];
        int best = 0, nonzero = 0;
        for (int k = 0; k < K; ++k) {
          if (cls[k] > cls[best]) best = k;
          nonzero += cls[k] > 0;
        }
        out->leaf_class[h] = best;
        pure = nonzero <= 1;
      }
      out->weight[h] = (double)nw;
      out->kind[h] = 0;
      if (depth == D || nw < 2 * (uint64_t)p->min_leaf || pure) continue;

      ora_split sp;
      uint32_t uid = (tree_id << 16) | (uint32_t)h;
      rc = ora_node_split(p, X, d, labels, y, nd->idx, nd->w, nd->n, uid, gbest,
                          NULL, &sp, NULL, NULL);
      if (rc) break;
      if (!sp.valid) continue;

      /* Partition, Eqs. (3)-(4): right (+) iff bin >= b*, i.e. z >= t_b. */
      int32_t* side = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nd->n > 0 ? nd->n : 1));
      if (!side) { rc = -2; break; }
      int64_t nl = 0;
      for (int64_t s = 0; s < nd->n; ++s) {
        int b = split_bin(p, gbest, sp.zmin, sp.inv_w, X + (int64_t)nd->idx[s] * d, d);
        side[s] = b >= sp.bin;
        nl += !side[s];
      }
      /* Zero gain: a split whose children keep the parent's class mix (or,
       * for MSE, does not lower the loss) is not made. */
      int no_gain = 0;
      if (p->criterion == ORA_MSE) {
        double sy = 0.0, sq = 0.0;
        for (int64_t s = 0; s < nd->n; ++s) {
          double ys = (double)y[nd->idx[s]];
          sy += (double)nd->w[s] * ys;
          sq += (double)nd->w[s] * ys * ys;
        }
        double parent = (sq - sy * sy / (double)nw) / (double)nw;
        no_gain = !(sp.loss < parent);
      } else {
        uint64_t* lk = (uint64_t*)calloc((size_t)K, sizeof(uint64_t));
        if (!lk) { free(side); rc = -2; break; }
        uint64_t wl = 0;
        for (int64_t s = 0; s < nd->n; ++s)
          if (!side[s]) {
            lk[labels[nd->idx[s]]] += nd->w[s];
            wl += nd->w[s];
          }
        no_gain = 1;
        for (int k = 0; k < K; ++k)
          if ((unsigned __int128)lk[k] * nw != (unsigned __int128)cls[k] * wl) no_gain = 0;
        free(lk);
      }
      if (no_gain) { free(side); continue; }

      out->kind[h] = 1;
      for (int32_t j = 0; j < d; ++j) out->dir[h * d + j] = gbest[j];
      out->zmin[h] = sp.zmin;
      out->inv_w[h] = sp.inv_w;
      out->bin[h] = sp.bin;
      out->loss[h] = sp.loss;
      out->n_left[h] = sp.n_left;
      out->n_right[h] = sp.n_right;

      int64_t nr = nd->n - nl;
      node_samples* L = &ns[2 * h + 1];
      node_samples* R = &ns[2 * h + 2];
      L->idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
      L->w = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(nl > 0 ? nl : 1));
      R->idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nr > 0 ? nr : 1));
      R->w = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(nr > 0 ? nr : 1));
      if (!L->idx || !L->w || !R->idx || !R->w) { free(side); rc = -2; break; }
      int64_t a = 0, c = 0;
      for (int64_t s = 0; s < nd->n; ++s) {
        if (side[s]) {
          R->idx[c] = nd->idx[s];
          R->w[c++] = nd->w[s];
        } else {
          L->idx[a] = nd->idx[s];
          L->w[a++] = nd->w[s];
        }
      }
      L->n = a;
      R->n = c;
      free(side);
    }
  }
  free(gbest);
  free(cls);

done:
  for (int64_t h = 0; h < H; ++h) {
    free(ns[h].idx);
    free(ns[h].w);
  }
  free(ns);
  return rc;
}

int ora_predict(const ora_params* p, const ora_tree* tree, const float* X,
                int64_t n, int32_t d, int32_t* class_out, double* value_out,
                int32_t* leaf_out) {
  if (!p || !tree || !X || d <= 0 || n < 0) return -1;
  const int64_t H = ((int64_t)1 << (p->max_depth + 1)) - 1;
  for (int64_t s = 0; s < n; ++s) {
    const float* xs = X + s * d;
    int64_t h = 0;
    while (h < H && tree->kind[h] == 1) {
      int b = split_bin(p, tree->dir + h * d, tree->zmin[h], tree->inv_w[h], xs, d);
      h = b >= tree->bin[h] ? 2 * h + 2 : 2 * h + 1;
    }
    if (class_out) class_out[s] = tree->leaf_class[h];
    if (value_out) value_out[s] = tree->leaf_value[h];
    if (leaf_out) leaf_out[s] = (int32_t)h;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* SLR Boost: least-squares gradient boosting of SLR trees on residuals.     */

int ora_train_boost(const ora_params* p, const float* X, int64_t n, int32_t d, const float* y,
                    int32_t M, float eta, ora_tree* trees, float* base_out, float* F,
                    double* mse_out) {
  if (!p || p->criterion != ORA_MSE || n < 1 || d < 1 || !X || !y || M < 0 ||
      !(eta > 0.0f && eta <= 1.0f) || !F || !base_out || (M > 0 && !trees))
    return -1;
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += (double)y[i];
  const float base = (float)(s / (double)n);
  float* r = (float*)malloc(sizeof(float) * (size_t)n);
  double* v = (double*)malloc(sizeof(double) * (size_t)n);
  int rc = 0;
  if (!r || !v) {
    rc = -2;
    goto done;
  }
  for (int64_t i = 0; i < n; ++i) F[i] = base;
  ora_params q = *p;
  for (int32_t m = 1; m <= M; ++m) {
    for (int64_t i = 0; i < n; ++i) r[i] = y[i] - F[i];
    q.seed = p->seed + (uint64_t)m;
    rc = ora_train_tree(&q, X, n, d, NULL, r, 0, 0, &trees[m - 1]);
    if (rc) goto done;
    rc = ora_predict(&q, &trees[m - 1], X, n, d, NULL, v, NULL);
    if (rc) goto done;
    for (int64_t i = 0; i < n; ++i) F[i] = F[i] + eta * (float)v[i];
    if (mse_out) {
      double e = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        const double di = (double)y[i] - (double)F[i];
        e += di * di;
      }
      mse_out[m - 1] = e / (double)n;
    }
  }
  *base_out = base;
done:
  free(r);
  free(v);
  return rc;
}

int ora_boost_predict(const ora_params* p, const ora_tree* trees, int32_t M, float base,
                      float eta, const float* X, int64_t n, int32_t d, float* out) {
  if (!p || M < 0 || (M > 0 && !trees) || !X || !out || n < 0 || d < 1) return -1;
  double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!v) return -2;
  int rc = 0;
  for (int64_t i = 0; i < n; ++i) out[i] = base;
  for (int32_t m = 0; m < M && !rc; ++m) {
    rc = ora_predict(p, &trees[m], X, n, d, NULL, v, NULL);
    for (int64_t i = 0; i < n && !rc; ++i) out[i] = out[i] + eta * (float)v[i];
  }
  free(v);
  return rc;
}

/* SLM Boost: K-class softmax gradient boosting with least-squares trees. */

/* Mean cross-entropy of F[n*K] against labels, in double. */
static double boost_ce(const float* F, const int32_t* labels, int64_t n, int32_t K) {
  double tot = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const float* f = F + i * K;
    double mx = (double)f[0];
    for (int32_t k = 1; k < K; ++k) mx = (double)f[k] > mx ? (double)f[k] : mx;
    double s = 0.0;
    for (int32_t k = 0; k < K; ++k) s += exp((double)f[k] - mx);
    tot += -(((double)f[labels[i]] - mx) - log(s));
  }
  return tot / (double)n;
}

void ora_softmax_residuals(const float* F, const int32_t* labels, int64_t n, int32_t K,
                           float* R) {
  for (int64_t i = 0; i < n; ++i) {
    const float* f = F + i * K;
    double mx = (double)f[0];
    for (int32_t k = 1; k < K; ++k) mx = (double)f[k] > mx ? (double)f[k] : mx;
    double s = 0.0;
    for (int32_t k = 0; k < K; ++k) s += exp((double)f[k] - mx);
    for (int32_t k = 0; k < K; ++k)
      R[(int64_t)k * n + i] = (float)((labels[i] == k ? 1.0 : 0.0) - exp((double)f[k] - mx) / s);
  }
}

int ora_train_boost_cls(const ora_params* p, const float* X, int64_t n, int32_t d,
                        const int32_t* labels, int32_t K, int32_t M, float eta,
                        ora_tree* trees, float* F, double* loss_out) {
  if (!p || n < 1 || d < 1 || !X || !labels || K < 2 || K > 64 || M < 0 ||
      !(eta > 0.0f && eta <= 1.0f) || !F || (M > 0 && !trees))
    return -1;
  for (int64_t i = 0; i < n; ++i)
    if (labels[i] < 0 || labels[i] >= K) return -1;
  float* R = (float*)malloc(sizeof(float) * (size_t)n * K);
  double* v = (double*)malloc(sizeof(double) * (size_t)n);
  int rc = 0;
  if (!R || !v) {
    rc = -2;
    goto done;
  }
  for (int64_t i = 0; i < n * K; ++i) F[i] = 0.0f;
  ora_params q = *p;
  q.criterion = ORA_MSE;
  q.n_classes = 0;
  for (int32_t m = 1; m <= M; ++m) {
    /* residuals of the softmax, all classes from the same F */
    ora_softmax_residuals(F, labels, n, K, R);
    /* the round's key is seed + m; class k's tree has tree id k (node uids
       (k << 16) | h), so the K trees of a round draw distinct streams */
    q.seed = p->seed + (uint64_t)m;
    for (int32_t k = 0; k < K; ++k) {
      ora_tree* t = &trees[(int64_t)(m - 1) * K + k];
      rc = ora_train_tree(&q, X, n, d, NULL, R + (int64_t)k * n, (uint32_t)k, 0, t);
      if (rc) goto done;
      rc = ora_predict(&q, t, X, n, d, NULL, v, NULL);
      if (rc) goto done;
      for (int64_t i = 0; i < n; ++i) F[i * K + k] = F[i * K + k] + eta * (float)v[i];
    }
    if (loss_out) loss_out[m - 1] = boost_ce(F, labels, n, K);
  }
done:
  free(R);
  free(v);
  return rc;
}

int ora_boost_predict_cls(const ora_params* p, const ora_tree* trees, int32_t M, int32_t K,
                          float eta, const float* X, int64_t n, int32_t d, float* F,
                          int32_t* class_out) {
  if (!p || M < 0 || K < 2 || (M > 0 && !trees) || !X || !F || n < 0 || d < 1) return -1;
  double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!v) return -2;
  ora_params q = *p;
  q.criterion = ORA_MSE;
  q.n_classes = 0;
  int rc = 0;
  for (int64_t i = 0; i < n * K; ++i) F[i] = 0.0f;
  for (int32_t m = 0; m < M && !rc; ++m)
    for (int32_t k = 0; k < K && !rc; ++k) {
      rc = ora_predict(&q, &trees[(int64_t)m * K + k], X, n, d, NULL, v, NULL);
      for (int64_t i = 0; i < n && !rc; ++i) F[i * K + k] = F[i * K + k] + eta * (float)v[i];
    }
  if (class_out && !rc)
    for (int64_t i = 0; i < n; ++i) {
      int32_t b = 0;
      for (int32_t k = 1; k < K; ++k)
        if (F[i * K + k] > F[i * K + b]) b = k;
      class_out[i] = b;
    }
  free(v);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Learned swarm proposal: node statistics, a 3-layer network, its loss and  */
/* gradient, Adam, and the seeded initial swarm. Written from the            */
/* definitions in slm_oracle.h, in double (the seeding in float).           */

int ora_node_stats(const float* X, int32_t d, const int32_t* labels,
                   int32_t n_classes, const float* y, const int32_t* idx,
                   const uint32_t* wts, int64_t n_idx, double* stats) {
  const int D = ORA_MLP_D, KM = ORA_MLP_K;
  if (!X || !idx || !stats || d < 1 || d > D || n_idx < 0) return -1;
  const int reg = labels == NULL;
  if (reg ? !y : (n_classes < 2 || n_classes > KM)) return -1;
  const int K = reg ? 4 : n_classes;
  for (int i = 0; i < ORA_MLP_IN; ++i) stats[i] = 0.0;
  float ylo = INFINITY, yhi = -INFINITY;
  if (reg)
    for (int64_t s = 0; s < n_idx; ++s) {
      float v = y[idx[s]];
      if (v < ylo) ylo = v;
      if (v > yhi) yhi = v;
    }
  double W = 0.0, Wk[ORA_MLP_K];
  double* sum = (double*)calloc((size_t)d, sizeof(double));
  double* csum = (double*)calloc((size_t)K * d, sizeof(double));
  if (!sum || !csum) {
    free(sum);
    free(csum);
    return -2;
  }
  for (int k = 0; k < K; ++k) Wk[k] = 0.0;
  for (int64_t s = 0; s < n_idx; ++s) {
    const double w = wts ? (double)wts[s] : 1.0;
    if (w == 0.0) continue;
    int k;
    if (reg) {
      /* quarter of the node's y range, in float, one rounding per operation */
      k = 0;
      if (yhi > ylo) {
        float f = 4.0f * ((y[idx[s]] - ylo) / (yhi - ylo));
        k = (int)floorf(f);
        if (k > 3) k = 3;
        if (k < 0) k = 0;
      }
    } else {
      k = labels[idx[s]];
    }
    const float* xs = X + (int64_t)idx[s] * d;
    W += w;
    Wk[k] += w;
    for (int j = 0; j < d; ++j) {
      sum[j] += w * (double)xs[j];
      csum[(int64_t)k * d + j] += w * (double)xs[j];
    }
  }
  if (W > 0.0) {
    for (int j = 0; j < d; ++j) sum[j] /= W; /* node mean */
    for (int64_t s = 0; s < n_idx; ++s) {
      const double w = wts ? (double)wts[s] : 1.0;
      const float* xs = X + (int64_t)idx[s] * d;
      for (int j = 0; j < d; ++j) {
        const double t = (double)xs[j] - sum[j];
        stats[(int64_t)KM * D + j] += w * t * t;
      }
    }
    for (int j = 0; j < d; ++j) stats[(int64_t)KM * D + j] /= W;
    for (int k = 0; k < K; ++k)
      if (Wk[k] > 0.0)
        for (int j = 0; j < d; ++j)
          stats[(int64_t)k * D + j] = csum[(int64_t)k * d + j] / Wk[k] - sum[j];
  }
  free(sum);
  free(csum);
  return 0;
}

/* weight as the network uses it: optionally rounded to bfloat16 */
static double mlp_w(double w, int bf16) {
  return bf16 ? (double)bf16_round((float)w) : w;
}

static void dense(const double* in, int n_in, const double* W, const double* b,
                  int n_out, int bf16, int relu, double* out) {
  for (int o = 0; o < n_out; ++o) {
    double acc = b[o];
    for (int i = 0; i < n_in; ++i) acc += in[i] * mlp_w(W[(int64_t)i * n_out + o], bf16);
    out[o] = relu && acc < 0.0 ? 0.0 : acc;
  }
}

int ora_mlp_forward(const ora_mlp* m, const double* s, int32_t n,
                    int32_t bf16_weights, double* h1, double* h2, double* out) {
  if (!m || !s || !out || n < 0) return -1;
  double* a1 = (double*)malloc(sizeof(double) * ORA_MLP_H);
  double* a2 = (double*)malloc(sizeof(double) * ORA_MLP_H);
  if (!a1 || !a2) {
    free(a1);
    free(a2);
    return -2;
  }
  for (int32_t r = 0; r < n; ++r) {
    dense(s + (int64_t)r * ORA_MLP_IN, ORA_MLP_IN, m->W1, m->b1, ORA_MLP_H, bf16_weights, 1, a1);
    dense(a1, ORA_MLP_H, m->W2, m->b2, ORA_MLP_H, bf16_weights, 1, a2);
    dense(a2, ORA_MLP_H, m->W3, m->b3, ORA_MLP_OUT, bf16_weights, 0,
          out + (int64_t)r * ORA_MLP_OUT);
    if (h1) memcpy(h1 + (int64_t)r * ORA_MLP_H, a1, sizeof(double) * ORA_MLP_H);
    if (h2) memcpy(h2 + (int64_t)r * ORA_MLP_H, a2, sizeof(double) * ORA_MLP_H);
  }
  free(a1);
  free(a2);
  return 0;
}

static double softplus(double x) { return x > 30.0 ? x : log1p(exp(x)); }
static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* Loss of one sample and dL/do (do[OUT]). */
static double sample_loss(const double* o, int dims, const double* a, double* dout) {
  const int D = ORA_MLP_D, P = ORA_MLP_P;
  double c = 0.0, mm = 0.0;
  for (int j = 0; j < dims; ++j) {
    c += o[j] * a[j];
    mm += o[j] * o[j];
  }
  const double q = mm + 1e-12;
  double loss = 1.0 - c * c / q;
  for (int j = 0; j < ORA_MLP_OUT; ++j) dout[j] = 0.0;
  for (int j = 0; j < dims; ++j) dout[j] = -2.0 * c * a[j] / q + 2.0 * c * c * o[j] / (q * q);
  /* distance of the unit prediction to the nearer of +-a */
  double delta = 1.0, nm = 0.0, sg = c >= 0.0 ? 1.0 : -1.0;
  if (mm > 0.0) {
    nm = sqrt(mm);
    double e = 0.0;
    for (int j = 0; j < dims; ++j) {
      const double t = o[j] / nm - sg * a[j];
      e += t * t;
    }
    delta = sqrt(e);
  }
  double spread = 0.0, dl_ddelta = 0.0;
  for (int i = 0; i < P; ++i) {
    const double tau = (i + 0.5) / P;
    const double x = o[D + i], rho = softplus(x), u = delta - rho;
    spread += u >= 0.0 ? tau * u : (tau - 1.0) * u;
    dl_ddelta += (u >= 0.0 ? tau : tau - 1.0) / P;
    const double dl_drho = (u >= 0.0 ? -tau : 1.0 - tau) / P;
    dout[D + i] = dl_drho * sigmoid(x);
  }
  /* d delta / d mu = (u - mu_hat (mu_hat . u)) / (|mu| delta), u = mu_hat - sg a */
  if (mm > 0.0 && delta > 0.0) {
    double hu = 0.0;
    for (int j = 0; j < dims; ++j) hu += (o[j] / nm) * (o[j] / nm - sg * a[j]);
    for (int j = 0; j < dims; ++j) {
      const double mh = o[j] / nm, uj = mh - sg * a[j];
      dout[j] += dl_ddelta * (uj - mh * hu) / (nm * delta);
    }
  }
  return loss + spread / P;
}

int ora_mlp_loss_grad(const ora_mlp* m, const double* s, const int32_t* dims,
                      const double* a, int32_t n, int32_t bf16_weights,
                      double* loss, double* gW1, double* gb1, double* gW2,
                      double* gb2, double* gW3, double* gb3) {
  const int IN = ORA_MLP_IN, H = ORA_MLP_H, OUT = ORA_MLP_OUT;
  if (!m || !s || !dims || !a || n < 1) return -1;
  for (int32_t r = 0; r < n; ++r)
    if (dims[r] < 1 || dims[r] > ORA_MLP_D) return -1;
  if (gW1) memset(gW1, 0, sizeof(double) * (size_t)IN * H);
  if (gb1) memset(gb1, 0, sizeof(double) * H);
  if (gW2) memset(gW2, 0, sizeof(double) * (size_t)H * H);
  if (gb2) memset(gb2, 0, sizeof(double) * H);
  if (gW3) memset(gW3, 0, sizeof(double) * (size_t)H * OUT);
  if (gb3) memset(gb3, 0, sizeof(double) * OUT);
  double* h1 = (double*)malloc(sizeof(double) * H);
  double* h2 = (double*)malloc(sizeof(double) * H);
  double* o = (double*)malloc(sizeof(double) * OUT);
  double* go = (double*)malloc(sizeof(double) * OUT);
  double* g2 = (double*)malloc(sizeof(double) * H);
  double* g1 = (double*)malloc(sizeof(double) * H);
  if (!h1 || !h2 || !o || !go || !g2 || !g1) {
    free(h1); free(h2); free(o); free(go); free(g2); free(g1);
    return -2;
  }
  double total = 0.0;
  const double inv_n = 1.0 / n;
  for (int32_t r = 0; r < n; ++r) {
    const double* sr = s + (int64_t)r * IN;
    dense(sr, IN, m->W1, m->b1, H, bf16_weights, 1, h1);
    dense(h1, H, m->W2, m->b2, H, bf16_weights, 1, h2);
    dense(h2, H, m->W3, m->b3, OUT, bf16_weights, 0, o);
    total += sample_loss(o, dims[r], a + (int64_t)r * ORA_MLP_D, go);
    for (int j = 0; j < OUT; ++j) go[j] *= inv_n;
    /* layer 3 */
    for (int i = 0; i < H; ++i) {
      double acc = 0.0;
      for (int j = 0; j < OUT; ++j) {
        if (gW3) gW3[(int64_t)i * OUT + j] += h2[i] * go[j];
        acc += mlp_w(m->W3[(int64_t)i * OUT + j], bf16_weights) * go[j];
      }
      g2[i] = h2[i] > 0.0 ? acc : 0.0;
    }
    if (gb3)
      for (int j = 0; j < OUT; ++j) gb3[j] += go[j];
    /* layer 2 */
    for (int i = 0; i < H; ++i) {
      double acc = 0.0;
      for (int j = 0; j < H; ++j) {
        if (gW2) gW2[(int64_t)i * H + j] += h1[i] * g2[j];
        acc += mlp_w(m->W2[(int64_t)i * H + j], bf16_weights) * g2[j];
      }
      g1[i] = h1[i] > 0.0 ? acc : 0.0;
    }
    if (gb2)
      for (int j = 0; j < H; ++j) gb2[j] += g2[j];
    /* layer 1 */
    if (gW1)
      for (int i = 0; i < IN; ++i)
        if (sr[i] != 0.0)
          for (int j = 0; j < H; ++j) gW1[(int64_t)i * H + j] += sr[i] * g1[j];
    if (gb1)
      for (int j = 0; j < H; ++j) gb1[j] += g1[j];
  }
  if (loss) *loss = total * inv_n;
  free(h1); free(h2); free(o); free(go); free(g2); free(g1);
  return 0;
}

void ora_adam_step(double* w, double* m, double* v, const double* g, int64_t n,
                   int32_t t, double lr, double beta1, double beta2, double eps) {
  const double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    w[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}

void ora_swarm_seed(uint64_t seed, uint32_t node_uid, int32_t P, int32_t d,
                    const float* mu_hat, const float* rho, float* pos) {
  float* u = (float*)malloc(sizeof(float) * (size_t)P * d);
  if (!u) return;
  ora_swarm_uniforms(seed, node_uid, 0, P, d, ORA_PURPOSE_SEED, u);
  const float sigma = sqrtf((float)d / 3.0f);
  for (int32_t i = 0; i < P; ++i) {
    float* ui = u + (int64_t)i * d;
    for (int32_t j = 0; j < d; ++j) ui[j] = 2.0f * ui[j] - 1.0f;
    float acc = 0.0f;
    for (int32_t j = 0; j < d; ++j) acc = fmaf(ui[j], ui[j], acc);
    const float nrm = sqrtf(acc);
    for (int32_t j = 0; j < d; ++j) {
      const float q = nrm > 0.0f ? ui[j] / nrm : 0.0f;
      pos[(int64_t)i * d + j] = sigma * (mu_hat[j] + rho[i] * q);
    }
  }
  free(u);
}
