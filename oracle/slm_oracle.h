/*
 * CPU oracle for SLM split search with particle swarm optimisation
 * (Fu et al., "Acceleration of Subspace Learning Machine via Particle Swarm
 * Optimization and Parallel Processing", arXiv 2208.07023).
 *
 * TEST INFRASTRUCTURE ONLY. This library is the correctness reference for the
 * CUDA implementation. Only the tests, the smoke check and the benchmark's CPU
 * baseline load it; the product path never calls it. It shares no code,
 * header, table or constant with the CUDA library.
 *
 * All arrays are row-major and live in host memory. Functions return 0 on
 * success and a negative number on bad arguments.
 */
#ifndef SLM_ORACLE_H
#define SLM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_GINI = 0, ORA_ENTROPY = 1, ORA_MSE = 2 };

/* Arithmetic mode of the projection, binning and swarm update.
 * ORA_F64:        every floating-point step in double precision.
 * ORA_F32_MIRROR: projection as a sequential fmaf over features, binning and
 *                 swarm update in float with one IEEE rounding per operation;
 *                 the criterion stays in double / exact integers.
 * ORA_BF16_TOPK:  every particle is first scored on a reduced-precision
 *                 projection: row and position rounded to bfloat16 (round to
 *                 nearest even), their dot product formed exactly and rounded
 *                 once to float. The `topk` particles with the lowest such
 *                 loss (ties to the lower index) are re-scored on the
 *                 ORA_F32_MIRROR projection. pbest takes the float score of
 *                 the re-scored particles and the bfloat16 score of the rest;
 *                 gbest is chosen among the re-scored particles only. Binning,
 *                 swarm update and partition follow ORA_F32_MIRROR. */
enum { ORA_F64 = 0, ORA_F32_MIRROR = 1, ORA_BF16_TOPK = 2 };

/* Philox stream purposes (high byte of counter word 3). */
enum {
  ORA_PURPOSE_INIT_X = 1,
  ORA_PURPOSE_INIT_V = 2,
  ORA_PURPOSE_R1 = 3,
  ORA_PURPOSE_R2 = 4,
  ORA_PURPOSE_BOOTSTRAP = 5,
  ORA_PURPOSE_SEED = 6
};

typedef struct {
  int32_t criterion;    /* ORA_GINI / ORA_ENTROPY / ORA_MSE */
  int32_t n_classes;    /* K >= 2 for classification, 0 for regression */
  int32_t n_particles;  /* P */
  int32_t n_iters;      /* T: swarm updates after the initial evaluation */
  int32_t n_bins;       /* B >= 2 */
  float inertia;        /* omega */
  float c1, c2;         /* learning factors */
  int32_t max_depth;    /* nodes at this depth are leaves */
  int32_t min_leaf;     /* >= 1, weighted sample count per child */
  uint64_t seed;        /* Philox key */
  int32_t precision;    /* ORA_F64 / ORA_F32_MIRROR / ORA_BF16_TOPK */
  int32_t n_threads;    /* 0: OpenMP default */
  int32_t topk;         /* ORA_BF16_TOPK: particles re-scored per evaluation */
  int32_t top_n;        /* 0 or >= d: every feature; else the swarm searches
                           the subspace of the node's top_n features by their
                           own split loss (ora_select_features) */
  int32_t apso;         /* 1: adaptive PSO (Sec. III-B): inertia, c1 and c2
                           set before every move by ora_apso_step, and in the
                           convergence state an elite candidate
                           (ora_elite_candidate) scored with the next
                           evaluation and applied by ora_elite_apply's rule.
                           Not with ORA_BF16_TOPK */
} ora_params;

/* Adaptive PSO (Sec. III-B; the rules of the cited APSO method): the
 * swarm's evolutionary state from the particles' mean distances, and the
 * inertia and learning factors of the next move. */
enum { ORA_APSO_EXPLORE = 1, ORA_APSO_EXPLOIT = 2, ORA_APSO_CONVERGE = 3,
       ORA_APSO_JUMPOUT = 4 };
enum { ORA_PURPOSE_APSO = 7 };
typedef struct {
  float f;       /* evolutionary factor (d_g - d_min) / (d_max - d_min) */
  int32_t state; /* ORA_APSO_* */
  float c1, c2;  /* learning factors of the next move */
  float w;       /* inertia of the next move */
} ora_apso;

/* One state update from positions x[P*d] (float values) and the index of
 * the particle that holds gbest: d_i = (sum over j != i, in increasing j, of
 * sqrtf of the sequential fmaf sum over features of (x_ik - x_jk)^2) / (P-1);
 * f = (d_g - d_min) / (d_max - d_min), 0 if d_max = d_min; the state from
 * f's fuzzy memberships (overlaps: keep prev_state if it is a candidate,
 * else the state after it in the ring 1 -> 2 -> 3 -> 4 -> 1, else the larger
 * membership, ties to the lower state); with delta in [0.05, 0.1]: explore
 * c1 += delta, c2 -= delta; exploit +0.5 delta, -0.5 delta; converge
 * +0.5 delta, +0.5 delta; jump out -delta, +delta; each clamped to [1.5,
 * 2.5], scaled by 4 / (c1 + c2) when the sum exceeds 4; w = 1 / (1 + 1.5
 * exp(-2.6 f)) in double, rounded to float. All float steps rounded once. */
void ora_apso_step(int32_t P, int32_t d, const double* x, int32_t gpart, int32_t prev_state,
                   float c1, float c2, float delta, ora_apso* out);

/* Elitist learning of the cited APSO method, candidate: gB with one
 * coordinate k moved by a Gaussian step. From the purpose-7 block at
 * (node_uid, t, 0, 0) with uniforms u0..u3 (lane 0 is the state update's
 * delta): k = floor(u1 d) (exact, in double); g = sqrt(-2 ln(1 - u2))
 * cos(2 pi u3) in double, rounded to float; sigma = 1 - 0.9 (t / T) in
 * float (the step's standard deviation falls linearly from 1 to 0.1 of the
 * initial range's width 2 over the search); e_k = gB_k + (2 sigma) g, in
 * float in the float modes. Writes e[d] and k. */
void ora_elite_candidate(uint64_t seed, uint32_t node_uid, uint32_t t, int32_t T, int32_t d,
                         const double* gb, int32_t precision, double* e, int32_t* k_out);

/* Elitist learning, acceptance, on losses (+inf: no admissible split; a
 * strictly lower loss is better): if the candidate's loss e_loss is below
 * gB's *g_loss, gB and the personal best of the gB particle gpart become the
 * candidate (position and loss); otherwise the particle with the worst
 * current loss (ties to the lower index) takes the candidate's position and
 * current loss, and its personal best too when the candidate beats it.
 * Arrays: x, pb [P*d]; cur_loss, pb_loss [P]; gb, elite [d]. Returns 1 when
 * accepted, else 0 with the replaced particle in *worst_out. */
int32_t ora_elite_apply(int32_t P, int32_t d, double* x, double* pb, double* cur_loss,
                        double* pb_loss, double* g_loss, int32_t gpart, double* gb,
                        const double* elite, double e_loss, int32_t* worst_out);

/* Result of scoring one projection vector on one node. */
typedef struct {
  double zmin, zmax, inv_w; /* projected range and bins per unit length */
  int32_t valid;            /* 0: no admissible threshold */
  int32_t bin;              /* best edge b in [1, B-1]: right iff bin >= b */
  double loss;              /* weighted child impurity; +inf if invalid */
  uint64_t q_num, q_den;    /* Gini only: Q = q_num / q_den, larger is better */
  double n_left, n_right;   /* weighted sample counts of the two children */
} ora_eval;

/* Result of a PSO split search on one node. */
typedef struct {
  int32_t valid;
  int32_t particle;         /* particle whose position became gbest last */
  int32_t iter_of_best;     /* iteration at which gbest last improved */
  int32_t bin;
  double zmin, inv_w;       /* binning of the gbest projection */
  double threshold;         /* zmin + bin / inv_w, in units of gB . x */
  double loss;
  uint64_t q_num, q_den;
  double n_left, n_right;
  int32_t first_near_tie;   /* first iteration at which another correct
                               implementation may take a different path: a
                               near-tie of double losses, or (ORA_BF16_TOPK) a
                               sample whose bfloat16 dot product is not exact
                               in float and lies near a bin edge; -1 if none */
  int32_t elite_tries;      /* adaptive PSO: elite candidates scored */
  int32_t elite_accepts;    /* ... of which became gB */
} ora_split;

/* Tree in heap layout: node h has children 2h+1 and 2h+2; H = 2^(D+1)-1. */
typedef struct {
  int32_t* kind;       /* [H] -1 absent, 0 leaf, 1 internal */
  double* dir;         /* [H*d] raw gbest position (not normalised) */
  double* zmin;        /* [H] */
  double* inv_w;       /* [H] */
  int32_t* bin;        /* [H] */
  int32_t* leaf_class; /* [H] majority class (classification) */
  double* leaf_value;  /* [H] mean target (regression) */
  double* weight;      /* [H] weighted sample count */
  double* loss;        /* [H] split loss (internal nodes) */
  double* n_left;      /* [H] */
  double* n_right;     /* [H] */
} ora_tree;

/* Philox4x32-10 block function (Salmon et al., SC'11). */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);

/* u[i*d + j] = uniform [0,1) draw of the swarm stream `purpose` for particle i,
 * dimension j at iteration t of node `node_uid`. */
void ora_swarm_uniforms(uint64_t seed, uint32_t node_uid, uint32_t t,
                        int32_t n_particles, int32_t d, int32_t purpose,
                        float* u);

/* Bootstrap multiplicities of tree `tree_id`: n draws with replacement. */
void ora_bootstrap(uint64_t seed, uint32_t tree_id, int64_t n, uint32_t* w);

/* One synchronous swarm update (Eq. pso-1, then x += v_new), in the mode's
 * precision. All arrays [P*d] except gbest [d]. */
void ora_pso_step(const ora_params* p, int32_t n_particles, int32_t d,
                  double* x, double* v, const double* pbest,
                  const double* gbest, const double* r1, const double* r2);

/* Score P projection vectors pos[P*d] on the node given by idx[n_idx]
 * (entry weights wts, NULL = 1). Optional outputs: bins_out[P*n_idx] and
 * z_out[P*n_idx] (particle-major). In ORA_BF16_TOPK mode bins / z are those
 * of the bfloat16 projection, and out[] holds the scores one search
 * iteration passes to pbest: the float re-score of the `topk` best particles
 * (none when topk == 0), the bfloat16 score of the others. */
int ora_eval_swarm(const ora_params* p, const float* X, int32_t d,
                   const int32_t* labels, const float* y, const int32_t* idx,
                   const uint32_t* wts, int64_t n_idx, const double* pos,
                   int32_t n_particles, ora_eval* out, int32_t* bins_out,
                   double* z_out);

/* Histogram and threshold scan of given bins (bins[s] in [0, B)) of the node
 * idx[n_idx]: fills valid, bin, loss, q_num, q_den, n_left, n_right of *out. */
int ora_score_bins(const ora_params* p, const int32_t* labels, const float* y,
                   const int32_t* idx, const uint32_t* wts, int64_t n_idx,
                   const int32_t* bins, ora_eval* out);

/* Round each float to the nearest bfloat16 (ties to even), returned as float. */
void ora_bf16_round(const float* in, float* out, int64_t n);

/* Feature pre-screen of one node (Sec. III-B, Algorithm 2): each feature k
 * scored as the projection on the unit vector e_k (z = x_k; float mirror or
 * double projection by p->precision, never bfloat16), the n best kept by the
 * particle ranking rule (better score, ties to the lower feature), returned
 * in increasing feature order in feat[n]. ev_out[d] (optional): every
 * feature's score; *near_tie (optional): the n-th and (n+1)-th scores are a
 * near-tie of double losses. */
int ora_select_features(const ora_params* p, const float* X, int32_t d,
                        const int32_t* labels, const float* y, const int32_t* idx,
                        const uint32_t* wts, int64_t n_idx, int32_t n, int32_t* feat,
                        ora_eval* ev_out, int32_t* near_tie);

/* PSO split search on one node (Algorithm 1 with synchronous updates).
 * With 0 < p->top_n < d the swarm searches the subspace of the node's top_n
 * features (ora_select_features; particle coordinate j is feature feat[j],
 * the same swarm streams as a d = top_n search) and the direction is lifted
 * back to d features with zeros elsewhere; a near-tie at the selection sets
 * first_near_tie = 0.
 * gbest_out[d]: raw position; dir_out[d]: gbest / ||gbest||;
 * trace_loss[T+1], trace_particle[T+1]: gbest after each evaluation. */
int ora_node_split(const ora_params* p, const float* X, int32_t d,
                   const int32_t* labels, const float* y, const int32_t* idx,
                   const uint32_t* wts, int64_t n_idx, uint32_t node_uid,
                   double* gbest_out, double* dir_out, ora_split* out,
                   double* trace_loss, int32_t* trace_particle);

/* ora_node_split (without the feature pre-screen) from a given initial
 * swarm: init_x[P*d] (float) replaces the uniform initial positions of Sec.
 * III-A, as a learned seed does; the velocities are the random start's. */
int ora_node_split_from(const ora_params* p, const float* X, int32_t d,
                        const int32_t* labels, const float* y, const int32_t* idx,
                        const uint32_t* wts, int64_t n_idx, uint32_t node_uid,
                        const float* init_x, double* gbest_out, double* dir_out,
                        ora_split* out, double* trace_loss, int32_t* trace_particle);

/* ---- probabilistic search (Sec. II-B: the projection search of the
 * original SLM, the baseline the swarm search replaces) -------------------
 * The node's features are ranked by their own split loss (each feature's
 * unit vector scored like any projection; better first, ties to the lower
 * feature): rank r (1-based) is feature rank_feat[r-1]. Each candidate
 * vector selects R of the D ranks and gives each selected rank r an integer
 * coefficient in [-floor(A_r), floor(A_r)], A_r = alpha0 exp(-alpha r)
 * (Eqs. dynamic, exp_a); the others are 0. */
enum { ORA_PURPOSE_PROB = 9 };
typedef struct {
  int32_t n_candidates;  /* I: candidates generated and scored */
  int32_t R;             /* coefficients selected per candidate, 1 <= R <= d */
  double gamma;          /* P_r: rank r is drawn with weight gamma^(r-1),
                            0 < gamma <= 1 (gamma^(r-1) by repeated products) */
  double alpha0, alpha;  /* the dynamic range A_r = alpha0 exp(-alpha r) */
  int32_t batch;         /* candidates per trace entry (>= 1) */
  int32_t q;             /* projections kept by the cosine pruning */
  int32_t cos_num, cos_den;  /* pruning threshold tau = cos_num / cos_den */
} ora_prob;

/* Candidate c of node node_uid: a_out[d] (integer values). Draw k is lane
 * k mod 4 of Philox4x32-10(seed, {node_uid, c, k / 4, 9 << 24}), as a
 * uniform u = (r >> 8) 2^-24. Draws 0..R-1 choose ranks without replacement:
 * target = u * (sum of the remaining ranks' weights, in rank order), the
 * first remaining rank whose running weight sum in rank order exceeds the
 * target (the last remaining one if none does). Draws R..2R-1 give the
 * chosen ranks' coefficients in order of choice: floor(u (2m + 1)) - m,
 * m = floor(A_r). All in double. */
void ora_prob_candidate(uint64_t seed, uint32_t node_uid, uint32_t c, int32_t d,
                        const int32_t* rank_feat, const ora_prob* pp, double* a_out);

/* The probabilistic search on one node: rank the features, score candidates
 * 0..I-1 with the projection arithmetic of p->precision (F64 or F32_MIRROR),
 * keep the best (strictly better replaces, so ties go to the lower
 * candidate). out: the best candidate's split (particle = its index,
 * iter_of_best = its batch); best_out[d]: its vector; trace_loss[ceil(I /
 * batch)] (optional): best loss after each batch; rank_feat_out[d]
 * (optional). Cosine pruning (diversity of the kept projections): repeatedly
 * the best candidate not yet pruned and not the zero vector is kept and
 * every candidate with cos^2 > tau^2 to it (exact integer test: cos_den^2
 * dot^2 > cos_num^2 |a|^2 |b|^2), itself included, is pruned, until q are
 * kept: kept[q] (optional), *n_kept. */
int ora_prob_search(const ora_params* p, const ora_prob* pp, const float* X, int32_t d,
                    const int32_t* labels, const float* y, const int32_t* idx,
                    const uint32_t* wts, int64_t n_idx, uint32_t node_uid, double* best_out,
                    ora_split* out, double* trace_loss, int32_t* rank_feat_out, int32_t* kept,
                    int32_t* n_kept);

/* Grow one tree (Algorithm 2, breadth-first). bootstrap != 0 draws the
 * tree's bag with ora_bootstrap(seed, tree_id, n). */
int ora_train_tree(const ora_params* p, const float* X, int64_t n, int32_t d,
                   const int32_t* labels, const float* y, uint32_t tree_id,
                   int32_t bootstrap, ora_tree* out);

/* ---- learned swarm proposal (a network that seeds the swarm) ------------
 * Fixed sizes: features padded to D = 256, classes to K = 20, P = 64 radii. */
enum {
  ORA_MLP_D = 256,
  ORA_MLP_K = 20,
  ORA_MLP_IN = 256 * 21,  /* 5376: K class blocks + one variance block */
  ORA_MLP_H = 512,
  ORA_MLP_P = 64,
  ORA_MLP_OUT = 256 + 64  /* direction, then P radii (before softplus) */
};

/* Network parameters, row-major, "input x output": W1[IN*H], b1[H],
 * W2[H*H], b2[H], W3[H*OUT], b3[OUT]. */
typedef struct {
  const double *W1, *b1, *W2, *b2, *W3, *b3;
} ora_mlp;

/* Statistics of one node (entries idx[n_idx], multiplicities wts or NULL),
 * the network input stats[IN]: block k < K (classes) holds, for j < d, the
 * class-k weighted mean of feature j minus the node's weighted mean (0 for an
 * empty class); block K holds the weighted (population) variance of feature j.
 * Regression (labels NULL): the classes are the four quarters of the node's
 * y range [ymin, ymax] (group = min(3, floor(4 (y - ymin) / (ymax - ymin)))). */
int ora_node_stats(const float* X, int32_t d, const int32_t* labels,
                   int32_t n_classes, const float* y, const int32_t* idx,
                   const uint32_t* wts, int64_t n_idx, double* stats);

/* Forward pass for n samples: h1 = relu(s W1 + b1), h2 = relu(h1 W2 + b2),
 * o = h2 W3 + b3. With bf16_weights, every weight (not bias) is rounded to
 * bfloat16 first. out[n*OUT]; h1, h2 (optional) [n*H]. */
int ora_mlp_forward(const ora_mlp* m, const double* s, int32_t n,
                    int32_t bf16_weights, double* h1, double* h2, double* out);

/* Mean loss over n samples and its gradient. For sample r with feature
 * count dims[r] and unit target direction a[r*D] (zero past dims[r]):
 * mu = o[0:dims], L_dir = 1 - (mu.a)^2 / (|mu|^2 + 1e-12); delta = |mu/|mu| -
 * sign(mu.a) a|; rho_i = softplus(o[D + i]); L_spread =
 * mean_i pinball_{tau_i}(delta - rho_i), tau_i = (i + 0.5) / P, pinball_tau(u)
 * = max(tau u, (tau - 1) u). Loss = mean_r (L_dir + L_spread). Gradients of
 * the loss (weights through the straight-through rule when bf16_weights):
 * g* arrays like the parameters; any may be NULL. */
int ora_mlp_loss_grad(const ora_mlp* m, const double* s, const int32_t* dims,
                      const double* a, int32_t n, int32_t bf16_weights,
                      double* loss, double* gW1, double* gb1, double* gW2,
                      double* gb2, double* gW3, double* gb3);

/* One Adam step (Kingma and Ba, 2015) on n parameters at step t >= 1:
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void ora_adam_step(double* w, double* m, double* v, const double* g, int64_t n,
                   int32_t t, double lr, double beta1, double beta2, double eps);

/* Seeded initial positions: x_i = sigma (mu_hat + rho_i u_i / |u_i|) with
 * u_ij = 2 U - 1 of the swarm stream (purpose ORA_PURPOSE_SEED = 6,
 * iteration 0) and sigma = sqrtf(d / 3.0f), the expected norm of a uniform
 * start in [-1, 1)^d, so that the start velocities 0.1 U[-1, 1) have the
 * same size relative to the positions as in a random start (the loss does
 * not depend on the scale of a direction); in float, one rounding per
 * operation; |u_i| = sqrtf of a sequential fmaf sum of squares. pos[P*d]. */
void ora_swarm_seed(uint64_t seed, uint32_t node_uid, int32_t n_particles,
                    int32_t d, const float* mu_hat, const float* rho, float* pos);

/* SLR Boost (Sec. V: the boosting ensemble of SLR trees), read as
 * least-squares gradient boosting: base = (float)(mean of y, summed in
 * double); F_i = base; for round m = 1..M: r_i = y_i - F_i (float), tree m
 * grown by ora_train_tree on (X, r) with the Philox key seed + m (tree id 0,
 * no bootstrap), F_i = F_i + eta * (float)v_i (float, rounded once per
 * operation) with v_i tree m's leaf value of x_i; mse_out[m-1] = mean over i
 * of (y_i - F_i)^2 in double after round m (may be NULL). trees[M] are
 * caller-allocated like ora_train_tree's; F[n] receives the final F.
 * Needs criterion ORA_MSE and 0 < eta <= 1. */
int ora_train_boost(const ora_params* p, const float* X, int64_t n, int32_t d, const float* y,
                    int32_t M, float eta, ora_tree* trees, float* base_out, float* F,
                    double* mse_out);

/* out[i] = base, then for m = 0..M-1: out[i] = out[i] + eta * (float)v_m(x_i). */
int ora_boost_predict(const ora_params* p, const ora_tree* trees, int32_t M, float base,
                      float eta, const float* X, int64_t n, int32_t d, float* out);

/* SLM Boost (Sec. V: the boosting ensemble of SLM trees), read as K-class
 * gradient boosting of the softmax cross-entropy with least-squares SLR
 * trees: F[i*K + k] = 0; round m = 1..M: in double, p_ik = exp(F_ik - max_j
 * F_ij) / (sum over j ascending of exp(F_ij - max_j F_ij)), and r_ik =
 * (float)([labels_i == k] - p_ik); then for k = 0..K-1 tree (m-1)*K + k is
 * grown by ora_train_tree (criterion ORA_MSE) on (X, r_.k) with the Philox
 * key seed + m and tree id k (node uids (k << 16) | h; no bootstrap: the K
 * trees of a round are a forest of K trees on K targets), and F_ik = F_ik +
 * eta * (float)v_ik (float). loss_out[m-1] (may be NULL): mean over i of
 * -log p_{i,labels_i} after round m, in double (log-sum-exp form).
 * trees[M*K] caller-allocated; p's criterion is ignored (trees use MSE). */
void ora_softmax_residuals(const float* F, const int32_t* labels, int64_t n, int32_t K,
                           float* R);  /* R[k*n + i], the residuals of one round */
int ora_train_boost_cls(const ora_params* p, const float* X, int64_t n, int32_t d,
                        const int32_t* labels, int32_t K, int32_t M, float eta,
                        ora_tree* trees, float* F, double* loss_out);

/* F[i*K + k] = 0 plus the rounds' eta * (float)v in round order; class_out[i]
 * = argmax over k of F_ik, ties to the lower class (either may be NULL). */
int ora_boost_predict_cls(const ora_params* p, const ora_tree* trees, int32_t M, int32_t K,
                          float eta, const float* X, int64_t n, int32_t d, float* F,
                          int32_t* class_out);

/* Route samples through a tree grown by ora_train_tree. */
int ora_predict(const ora_params* p, const ora_tree* tree, const float* X,
                int64_t n, int32_t d, int32_t* class_out, double* value_out,
                int32_t* leaf_out);

#ifdef __cplusplus
}
#endif
#endif
