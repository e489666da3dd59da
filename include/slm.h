/*
 * libslm -- GB300 (sm_103a) split search for the Subspace Learning Machine
 * with particle swarm optimisation (Fu et al., arXiv 2208.07023).
 *
 * The problem (Sec. II-A, Eqs. 1-4): at a tree node, find a direction a and a
 * threshold t_b such that the half-spaces a^T x >= t_b (right, "+") and
 * a^T x < t_b (left, "-") have the lowest weighted child impurity. The
 * direction is searched by a particle swarm (Sec. III-A, Eq. pso-1,
 * Algorithm 1); each particle's projection is scored by binning it into B
 * uniform bins on [min z, max z] and scanning the B-1 interior bin edges as
 * thresholds (the paper's "loss at each split point", Sec. IV). Trees grow by
 * repeating the search on the children (Algorithm 2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory.    Array arguments may be device pointers or host pointers; the
 *            library inspects each with cudaPointerGetAttributes. Host inputs
 *            are staged to the device and host outputs copied back inside the
 *            call. Every array is row-major and dense.
 * Ownership. The caller owns every buffer it passes and may free it when the
 *            call returns, except that slm_forest_begin keeps X / labels / y
 *            (if device pointers) until slm_forest_free. Forests are owned by
 *            the library and released with slm_forest_free.
 * Streams.   Work is issued on the context's stream. Calls that return host
 *            results synchronise that stream before returning.
 * Errors.    Every entry point returns an slm_status; no C++ exception
 *            crosses this boundary. SLM_EINVAL: an argument is out of range
 *            (nothing was launched). SLM_ECUDA: a CUDA call failed; the
 *            message is available from slm_last_error. SLM_EUNSUPPORTED: the
 *            sizes are valid but exceed a compiled limit listed below.
 * Threads.   A context may be used by one host thread at a time.
 * Limits.    1 <= d <= 1024; 1 <= P (n_particles) <= 256; 2 <= B (n_bins) <= 256;
 *            2 <= K (n_classes) <= 32; 0 <= max_depth <= 15; n < 2^31;
 *            per-particle histogram B*K*4 bytes <= 10240 (classification).
 *            SLM_PROJ_BF16_TOPK: round16(P) * round16(d) * 2 <= 131072.
 */
#ifndef SLM_H
#define SLM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SLM_OK = 0,
  SLM_EINVAL = 1,
  SLM_ENOMEM = 2,
  SLM_ECUDA = 3,
  SLM_ETIMEOUT = 4,
  SLM_EUNSUPPORTED = 5
} slm_status;

/* Child impurity (Sec. II-A: "lower entropy"; Table 4 reports MSE).
 * GINI:    loss = sum_side (n_side/n) (1 - sum_k p_k^2).
 * ENTROPY: loss = sum_side (n_side/n) (-sum_k p_k ln p_k), natural log.
 * MSE:     loss = (SSE_left + SSE_right) / n. */
typedef enum { SLM_GINI = 0, SLM_ENTROPY = 1, SLM_MSE = 2 } slm_criterion;

/* Projection arithmetic. FP32: z = sum_j x_j a_j as one fused multiply-add
 * per feature in increasing j, starting from +0.
 * BF16_TOPK: every particle is first scored on z~ = sum_j bf16(x_j) bf16(a_j)
 * (bfloat16 operands rounded to nearest even, exact products, FP32
 * accumulation in the tensor cores' order); per node the `topk` particles
 * with the best such score (ties to the lower index) are re-scored on the
 * FP32 projection. pbest takes the FP32 score of a re-scored particle and the
 * bfloat16 score of the others; gbest is chosen among the re-scored
 * particles only, so every gB score and every split is an FP32 score. This
 * mode is not in the paper: it trades the projection's precision for tensor-
 * core throughput and keeps the split decisions in FP32. */
typedef enum { SLM_PROJ_FP32 = 0, SLM_PROJ_BF16_TOPK = 1 } slm_proj;

typedef struct slm_params {
  int32_t criterion;   /* slm_criterion */
  int32_t n_classes;   /* K for GINI / ENTROPY; 0 for MSE */
  int32_t n_particles; /* P: swarm size (Eq. pso_a) */
  int32_t n_iters;     /* T: swarm updates after the initial evaluation */
  int32_t n_bins;      /* B: uniform bins per projection */
  int32_t topk;        /* SLM_PROJ_BF16_TOPK: particles re-scored in FP32 per
                          node and iteration, 1..P (slm_evaluate_swarm: 0..P,
                          0 = none); unused otherwise */
  float inertia;       /* omega in Eq. pso-1 */
  float c1, c2;        /* learning factors in Eq. pso-1 */
  int32_t max_depth;   /* nodes at this depth are leaves */
  int32_t min_leaf;    /* >= 1: minimum weighted samples in each child */
  int32_t proj;        /* slm_proj */
  int32_t n_trees;     /* >= 1; > 1 grows a bagged forest */
  int32_t bootstrap;   /* 1: tree t trains on a bootstrap bag of the n samples */
  int32_t seeded;      /* 1: start each swarm from the context's proposal
                          (slm_use_proposal) instead of U[-1,1)^d; 0 otherwise */
  int32_t top_n;       /* 0 or >= d: the swarm searches all d features.
                          0 < top_n < d (Sec. III-B, Algorithm 2: features
                          pre-screened per node): every feature k of a node
                          is first scored on its own (the projection on the
                          unit vector e_k, scored like a particle), the
                          top_n best are kept (better score, ties to the
                          lower feature; in increasing feature order), the
                          swarm searches their subspace (coordinate j is the
                          j-th kept feature; the swarm streams of a top_n-
                          dimensional search) and gB is returned lifted to d
                          features, zero elsewhere. Needs SLM_PROJ_FP32,
                          seeded = 0 and d <= 256 (SLM_EUNSUPPORTED) */
  int32_t apso;        /* 1: adaptive PSO (Sec. III-B, with the published
                          rules of the cited APSO method): before every move
                          each node's evolutionary state is estimated from
                          the particles' mean distances and the move uses
                          the state's learning factors (from c1, c2 at the
                          start) and an inertia from the evolutionary factor
                          (inertia is then unused); in the convergence state
                          a copy of gB with one coordinate moved by a
                          Gaussian step is scored with the next evaluation
                          and replaces gB if better, else the worst
                          particle (elitist learning); 0: plain PSO. Needs
                          SLM_PROJ_FP32 and n_particles < 256 with
                          (n_particles rounded up to 4) * d * 4 <= 200 KB
                          (SLM_EUNSUPPORTED) */
  uint64_t seed;       /* Philox-4x32-10 key for every random draw */
} slm_params;

/* Score of one projection vector on one node (the best of its B-1 edges). */
typedef struct slm_eval {
  double loss;         /* +inf if no admissible edge */
  uint64_t q_num;      /* GINI only: Q = q_num / q_den = S_L/n_L + S_R/n_R; */
  uint64_t q_den;      /*   loss = 1 - Q/n; larger Q is strictly better */
  float zmin, inv_w;   /* bin(z) = min(B-1, floor((z - zmin) * inv_w)) */
  int32_t bin;         /* best edge b in [1, B-1]; right child iff bin(z) >= b */
  int32_t valid;       /* 0: all projections equal, or no edge leaves
                          min_leaf samples on both sides */
  int64_t n_left;      /* weighted sample counts of the children */
  int64_t n_right;
} slm_eval;

/* Result of a PSO split search on one node (Algorithm 1). */
typedef struct slm_split {
  slm_eval eval;       /* score of the global best position gB */
  int32_t particle;    /* particle whose position became gB last */
  int32_t iter_of_best;/* iteration at which gB last improved (0 = init) */
  float threshold;     /* zmin + bin / inv_w, in units of gB . x */
  float norm;          /* ||gB||: t_b for the unit direction is threshold/norm */
} slm_split;

typedef struct slm_ctx slm_ctx;
typedef struct slm_forest slm_forest;

const char* slm_status_string(slm_status s);

/* Creates a context on `device` issuing work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream). */
slm_status slm_create(slm_ctx** out, int device, void* cuda_stream);
void slm_destroy(slm_ctx* ctx);
/* Copies the last error message (NUL-terminated, truncated to len). */
slm_status slm_last_error(slm_ctx* ctx, char* buf, size_t len);

/* Uniform [0,1) draws of the swarm streams (Sec. III-A: random initial
 * positions and velocities, r1 and r2 of Eq. pso-1), exposed for
 * reproducibility checks. u[i*d + j] = (r >> 8) * 2^-24 with r = lane (j mod 4)
 * of Philox4x32-10(key = seed, counter = {node_uid, t, i, (j>>2) | purpose<<24}).
 * purpose: 1 initial position, 2 initial velocity, 3 r1, 4 r2, 6 seeded
 * start (slm_swarm_seed). */
slm_status slm_swarm_uniforms(slm_ctx* ctx, uint64_t seed, uint32_t node_uid,
                              uint32_t t, int32_t n_particles, int32_t d,
                              int32_t purpose, float* u);

/* Bootstrap multiplicities of tree `tree_id` (Sec. V, SLM Forest): n draws
 * with replacement, draw k = floor(r * n / 2^32) with r = lane (k mod 4) of
 * Philox4x32-10(seed, {tree_id, k>>2, 0, 5<<24}). w[n] receives the counts. */
slm_status slm_bootstrap(slm_ctx* ctx, uint64_t seed, uint32_t tree_id,
                         int64_t n, uint32_t* w);

/* Scores n_pos projection vectors (rows of positions[n_pos*d]) on one node:
 * the node holds rows sample_idx[0..n_idx) of X[n*d] (sample_idx NULL = all
 * n rows) with multiplicities weights[n_idx] (NULL = 1). Exactly one of
 * labels[n] (classification) and y[n] (MSE) is non-NULL. out[n_pos] is
 * written; bins_out[n_pos*n_idx] (optional) receives bin(z) per particle and
 * node entry. Uses params: criterion, n_classes, n_bins, min_leaf, proj,
 * topk. With SLM_PROJ_BF16_TOPK, bins_out holds the bfloat16 projection's
 * bins and out[] the scores one search iteration passes to pbest: the FP32
 * re-score of the topk best particles, the bfloat16 score of the others. */
slm_status slm_evaluate_swarm(slm_ctx* ctx, const slm_params* params,
                              const float* X, int64_t n, int32_t d,
                              const int32_t* labels, const float* y,
                              const int32_t* sample_idx,
                              const uint32_t* weights, int64_t n_idx,
                              const float* positions, int32_t n_pos,
                              slm_eval* out, int32_t* bins_out);

/* Size of the fixed device array behind slm_evaluate_swarm_noalloc. */
#define SLM_NOALLOC_SCRATCH_BYTES (32u << 20)

/* slm_evaluate_swarm for callers that must not allocate device memory: code
 * whose device memory is reserved up front and then handed out by its own
 * pool (a host application or plugin framework that forbids cudaMalloc
 * inside its work loop, since an allocation can block, synchronise the
 * device or fail once memory is committed), or code running where the
 * caching allocator is unavailable. The paper has no counterpart to this
 * entry point.
 *
 * It performs no cudaMalloc / cudaFree and calls no allocating library
 * routine. Its scratch is one fixed array of SLM_NOALLOC_SCRATCH_BYTES in the
 * library's device memory, which every GPU that loads the library holds until
 * the process exits. A call needs about 4 * (n_idx * (d + n_pos + 4) + P' * d)
 * bytes of it, P' = n_pos rounded up to a multiple of 16, plus 16 * n_idx for
 * MSE (each part rounded up to 256 bytes); larger calls return
 * SLM_EUNSUPPORTED and do nothing.
 *
 * Same meaning as slm_evaluate_swarm with params->proj = SLM_PROJ_FP32
 * (this entry point scores with the FP32 projection only:
 * SLM_PROJ_BF16_TOPK returns SLM_EUNSUPPORTED, an unknown proj SLM_EINVAL),
 * except: X, labels / y, sample_idx, weights and positions must be device
 * (or managed) memory of `device`, and out[n_pos] is a device buffer the call
 * fills; a host or another GPU's pointer returns SLM_EINVAL before anything
 * is launched. Work runs on `cuda_stream` of `device`; the call synchronises
 * that stream twice (it reads a validation word and the kernels' error word
 * back) and returns after the stream has finished its work. The calling
 * thread's current device is restored before the call returns. The first
 * call on a device looks up the array's device address (once per device);
 * make that first call before any stream capture. Every call overwrites the
 * array (the call resets what must start fresh), so calls whose work
 * overlaps on the GPU -- on other streams or from other host threads -- race
 * and must be serialised by the caller. Errors: SLM_EINVAL bad arguments,
 * pointers, labels or sample indices; SLM_EUNSUPPORTED sizes beyond the
 * array or the BF16 form; SLM_ECUDA a CUDA call failed or a kernel reported
 * an error; SLM_ETIMEOUT a staged copy did not complete. */
slm_status slm_evaluate_swarm_noalloc(int device, void* cuda_stream,
                                      const slm_params* params, const float* X,
                                      int64_t n, int32_t d,
                                      const int32_t* labels, const float* y,
                                      const int32_t* sample_idx,
                                      const uint32_t* weights, int64_t n_idx,
                                      const float* positions, int32_t n_pos,
                                      slm_eval* out);

/* PSO split search on one node (Algorithm 1, synchronous updates: every
 * particle moves with the gB held at the end of the previous iteration; pB
 * and gB change only on a strictly lower loss, ties to the lower particle
 * index). node_uid keys the node's Philox streams. direction_out[d]: gB/||gB||
 * (Eq. 2); gbest_out[d] (optional): gB itself, on which bin(z) is defined;
 * trace_out[T+1] (optional): gB loss after each evaluation. */
slm_status slm_node_split(slm_ctx* ctx, const slm_params* params,
                          const float* X, int64_t n, int32_t d,
                          const int32_t* labels, const float* y,
                          const int32_t* sample_idx, const uint32_t* weights,
                          int64_t n_idx, uint32_t node_uid,
                          float* direction_out, float* gbest_out,
                          slm_split* out, double* trace_out);

/* Tree / forest growth (Algorithm 2), level by level. Each call to
 * slm_grow_level searches every splittable node of the current level of
 * every tree in one batch (node uid = tree_id << 16 | heap index) and
 * partitions their samples into the next level. A node is a leaf when it is
 * at max_depth, holds < 2*min_leaf weighted samples, is pure (one class /
 * constant target), has no admissible split, or its best split does not lower
 * the impurity. *n_split_out (optional) = nodes split by this call; 0 means
 * the forest is complete. */
slm_status slm_forest_begin(slm_ctx* ctx, const slm_params* params,
                            const float* X, int64_t n, int32_t d,
                            const int32_t* labels, const float* y,
                            slm_forest** out);
slm_status slm_grow_level(slm_ctx* ctx, slm_forest* forest,
                          int32_t* n_split_out);
/* Probabilistic search (Sec. II-B: the projection search of the original
 * SLM, which the swarm search replaces; kept as a baseline). The node's
 * features are ranked by their own split loss (each unit vector scored like
 * a projection; better first, ties to the lower feature). Each of
 * n_candidates vectors selects R of the d ranks without replacement, rank r
 * (1-based) with weight gamma^(r-1) (the exponentially falling P_d), and
 * gives each an integer coefficient drawn uniformly from -m_r .. m_r,
 * m_r = floor(alpha0 exp(-alpha r)) (Eqs. dynamic, exp_a); the other
 * coefficients are 0. Draw k of candidate c is lane k mod 4 of
 * Philox4x32-10(seed, {node_uid, c, k / 4, 9 << 24}) as (r >> 8) 2^-24:
 * draws 0..R-1 choose ranks (target u * (sum of the remaining weights), the
 * first remaining rank, in rank order, whose running weight sum passes it),
 * draws R..2R-1 the chosen ranks' coefficients, floor(u (2 m + 1)) - m, in
 * double. Candidates are scored in batches of `batch` like swarm particles
 * (FP32 projection) and the best is kept (a later candidate replaces it only
 * when strictly better). Cosine pruning keeps up to q diverse projections:
 * repeatedly the best candidate not yet pruned and not zero, then every
 * candidate b with cos_den^2 (a.b)^2 > cos_num^2 |a|^2 |b|^2 to it (exact
 * integers) is pruned, itself included. */
typedef struct {
  int32_t n_candidates;  /* 1 .. 2^20 */
  int32_t R;             /* 1 .. min(d, 64) */
  double gamma;          /* (0, 1] */
  double alpha0, alpha;  /* 0 <= alpha0 <= 100, alpha >= 0 */
  int32_t batch;         /* 1 .. 256: candidates per scoring pass and trace entry */
  int32_t q;             /* >= 0 */
  int32_t cos_num, cos_den;  /* 0 <= cos_num <= cos_den <= 100, cos_den >= 1 */
} slm_prob;
/* On one node (arguments as slm_node_split; params: criterion, n_classes,
 * n_bins, min_leaf, seed, proj = SLM_PROJ_FP32): *out the best candidate's
 * split (particle = its index, iter_of_best = its batch), best_out[d]
 * (optional) its vector, direction_out[d] the vector normalised;
 * trace_out[ceil(n_candidates / batch)] (optional) the best loss after each
 * batch; rank_feat_out[d] (optional) the features in rank order;
 * kept_out[q] (optional) and *n_kept_out (optional) the pruning's kept
 * candidates. SLM_EINVAL for arguments outside the ranges above. */
slm_status slm_prob_search(slm_ctx* ctx, const slm_params* params, const slm_prob* prob,
                           const float* X, int64_t n, int32_t d, const int32_t* labels,
                           const float* y, const int32_t* sample_idx, const uint32_t* weights,
                           int64_t n_idx, uint32_t node_uid, float* direction_out,
                           float* best_out, slm_split* out, double* trace_out,
                           int32_t* rank_feat_out, int32_t* kept_out, int32_t* n_kept_out);

/* Global tree ids of the forests the context begins from now on: local
 * tree t of a forest is tree first + t * stride of a larger forest, whose
 * bootstrap draw (slm_bootstrap, tree_id) and node uids (tree_id << 16 |
 * heap index) it uses, so that N processes growing trees r, r + N, ... of
 * one forest (Sec. V, SLM Forest) with first = r, stride = N together grow
 * exactly the trees one process would. Defaults 0, 1. SLM_EINVAL unless
 * 0 <= first <= 65535 and 1 <= stride <= 65535; a forest whose ids would
 * pass 65535 is refused by slm_forest_begin. */
slm_status slm_set_tree_ids(slm_ctx* ctx, int64_t first, int64_t stride);
/* forest_begin + grow_level until complete. */
slm_status slm_train_tree(slm_ctx* ctx, const slm_params* params,
                          const float* X, int64_t n, int32_t d,
                          const int32_t* labels, const float* y,
                          slm_forest** out);
void slm_forest_free(slm_forest* forest);

/* Number of trees, heap size H = 2^(max_depth+1) - 1, feature count, and the
 * particle-sample evaluations performed so far: the sum over searched nodes
 * of (distinct samples in the node) * P * (T+1). Any pointer may be NULL. */
slm_status slm_forest_info(const slm_forest* forest, int32_t* n_trees,
                           int32_t* heap_size, int32_t* d,
                           int64_t* evaluations);

/* Copies tree `tree` of a forest to host arrays in heap layout (node h has
 * children 2h+1 and 2h+2); any pointer may be NULL. kind: -1 absent, 0 leaf,
 * 1 internal. dir[H*d]: raw gB of the split. leaf_class / leaf_value: majority
 * class (ties to the lowest id) / mean target. */
slm_status slm_forest_export(slm_ctx* ctx, const slm_forest* forest,
                             int32_t tree, int32_t* kind, float* dir,
                             float* zmin, float* inv_w, int32_t* bin,
                             int32_t* leaf_class, double* leaf_value,
                             int64_t* weight, double* loss, int64_t* n_left,
                             int64_t* n_right);

/* Routes X[n*d] through every tree: internal node h sends x right iff
 * bin_h(gB_h . x) >= bin_h, with bin clamped to [0, B-1]. class_out[n]
 * (classification): majority vote over trees, ties to the lowest class;
 * value_out[n] (MSE): mean of the trees' leaf values; leaf_out[n*n_trees]
 * (optional): heap index of the leaf reached in each tree. */
slm_status slm_predict(slm_ctx* ctx, const slm_forest* forest, const float* X,
                       int64_t n, int32_t d, int32_t* class_out,
                       double* value_out, int32_t* leaf_out);


/* ---- SLR / SLM Boost -----------------------------------------------------
 * The boosting ensembles of SLR and SLM trees (Sec. V names SLR Boost and SLM
 * Boost beside the forests), read as gradient boosting with least-squares
 * SLR trees on residuals, in float. Regression (y):
 *   base = (float)(mean of y, summed in double);  F_i = base;
 *   round m = 1..n_rounds: r_i = y_i - F_i; one SLR tree grown on (X, r)
 *   with `params` and the Philox key params->seed + m (tree id 0);
 *   F_i = F_i + learning_rate * (float)v_i, v_i the tree's leaf value of x_i.
 * Classification (labels, K = params->n_classes classes): F_ik = 0; round m:
 *   in double p_ik = exp(F_ik - max_j F_ij) / sum_j (ascending) of the same,
 *   r_ik = (float)([labels_i == k] - p_ik) (all k from the same F); the
 *   K trees of the round, tree k on (X, r_.k), grown together as one forest
 *   (every level of all K searched in one batch) with the key params->seed
 *   + m and tree ids 0..K-1 (node uids (k << 16) | h); then for k =
 *   0..K-1 F_ik = F_ik + learning_rate * (float)v_ik.
 * Each float operation is rounded once. */
typedef struct slm_boost slm_boost;

/* Trains n_rounds >= 0 rounds on X[n*d] and exactly one of labels[n] (values
 * in [0, K), 2 <= K <= 32) and y[n] (host or device; host inputs are
 * copied). params: criterion SLM_MSE (the trees fit residuals), n_trees 1,
 * bootstrap 0 (SLM_EINVAL / SLM_EUNSUPPORTED otherwise); 0 < learning_rate
 * <= 1. train_loss_out[n_rounds] (host or device, may be NULL): after each
 * round, in double, the mean of (y - F)^2, or the mean cross-entropy
 * -log p_{i, labels_i} (log-sum-exp form). On success *out owns the trees
 * (slm_boost_free). */
slm_status slm_train_boost(slm_ctx* ctx, const slm_params* params, const float* X,
                           int64_t n, int32_t d, const int32_t* labels, const float* y,
                           int32_t n_rounds, float learning_rate, double* train_loss_out,
                           slm_boost** out);
/* value_out[n * n_outputs] (may be NULL): the scores F (base for regression,
 * 0 for classification, plus the rounds' learning_rate * (float) leaf values
 * in round order: the training F for the training rows); class_out[n]
 * (classification, may be NULL): argmax over k of F_ik, ties to the lower
 * class. Host or device pointers. */
slm_status slm_boost_predict(slm_ctx* ctx, const slm_boost* boost, const float* X,
                             int64_t n, int32_t d, float* value_out, int32_t* class_out);
/* Rounds, outputs (1 or K), base (regression) and learning rate; any
 * pointer may be NULL. */
slm_status slm_boost_info(const slm_boost* boost, int32_t* n_rounds, int32_t* n_outputs,
                          float* base, float* learning_rate);
/* Tree t = m * n_outputs + k (round m + 1, output k), owned by the boost
 * (read it with slm_forest_export / slm_predict; do not free it); NULL if t
 * is out of range. */
const slm_forest* slm_boost_tree(const slm_boost* boost, int32_t t);
void slm_boost_free(slm_boost* boost);

/* ---- learned swarm proposal ----------------------------------------------
 * Not in the paper, which starts every swarm uniformly in a fixed range (Sec. III-A):
 * a network that proposes a starting direction and spread for a node's swarm
 * from the node's statistics, trained on (statistics, best direction) pairs
 * that PSO searches produce. Sizes are fixed: features padded to
 * SLM_PROPOSAL_D, classes to SLM_PROPOSAL_K, SLM_PROPOSAL_P spread radii. */
#define SLM_PROPOSAL_D 256
#define SLM_PROPOSAL_K 20
#define SLM_PROPOSAL_IN (256 * 21)  /* 5376 statistics per node */
#define SLM_PROPOSAL_H 512          /* hidden width */
#define SLM_PROPOSAL_P 64
#define SLM_PROPOSAL_OUT (256 + 64) /* direction, then radii before softplus */

typedef struct slm_proposal slm_proposal;

/* Statistics of one node, the network input stats[SLM_PROPOSAL_IN] (host or
 * device): for class k < K and feature j < d, stats[k*256 + j] = the class's
 * weighted mean of feature j minus the node's (0 for an empty class);
 * stats[20*256 + j] = the node's weighted variance of feature j; all other
 * entries 0. Regression (labels NULL, y set): the classes are the quarters of
 * the node's y range. Node and weights as in slm_evaluate_swarm. Limits:
 * d <= 256, n_classes <= 20. */
slm_status slm_node_stats(slm_ctx* ctx, const float* X, int64_t n, int32_t d,
                          const int32_t* labels, int32_t n_classes,
                          const float* y, const int32_t* sample_idx,
                          const uint32_t* weights, int64_t n_idx,
                          float* stats);

/* A network h1 = relu(s W1 + b1), h2 = relu(h1 W2 + b2), o = h2 W3 + b3 with
 * W1[IN x H], W2[H x H], W3[H x OUT] row-major ("input x output"), computed
 * with bfloat16-rounded weights and FP32 accumulation. Created with
 * Glorot-uniform weights from Philox (seed) and zero biases; owned by the
 * library, freed by slm_proposal_free. */
slm_status slm_proposal_create(slm_ctx* ctx, uint64_t seed, slm_proposal** out);
void slm_proposal_free(slm_proposal* prop);
/* Copies all parameters in (set: also resets the Adam state) or out; arrays
 * are FP32, host or device, any may be NULL on get. */
slm_status slm_proposal_set(slm_ctx* ctx, slm_proposal* prop, const float* W1,
                            const float* b1, const float* W2, const float* b2,
                            const float* W3, const float* b3);
slm_status slm_proposal_get(slm_ctx* ctx, const slm_proposal* prop, float* W1,
                            float* b1, float* W2, float* b2, float* W3,
                            float* b3);
/* out[N x OUT] = network(stats[N x IN]). */
slm_status slm_proposal_forward(slm_ctx* ctx, const slm_proposal* prop,
                                const float* stats, int32_t n, float* out);
/* Mean loss over n samples and its gradient (g* like the parameters, FP32,
 * host or device, any may be NULL). Sample r: d = dims[r] features, unit
 * target direction targets[r*256 ...] (zero past d); mu = o[0:d],
 * L = 1 - (mu.a)^2 / (|mu|^2 + 1e-12) + mean_i pinball_{(i+0.5)/64}(delta -
 * softplus(o[256+i])), delta = |mu/|mu| - sign(mu.a) a|. Gradients pass
 * straight through the bfloat16 rounding of the weights. */
slm_status slm_proposal_loss_grad(slm_ctx* ctx, const slm_proposal* prop,
                                  const float* stats, const int32_t* dims,
                                  const float* targets, int32_t n, double* loss,
                                  float* gW1, float* gb1, float* gW2, float* gb2,
                                  float* gW3, float* gb3);
/* Trains with Adam (lr, beta 0.9 / 0.999, eps 1e-8) on n samples for
 * `epochs` passes in minibatches of `batch` (order shuffled per epoch from
 * `seed`); epoch_loss[epochs] (optional, host) receives each epoch's mean
 * batch loss. */
slm_status slm_proposal_train(slm_ctx* ctx, slm_proposal* prop,
                              const float* stats, const int32_t* dims,
                              const float* targets, int32_t n, int32_t epochs,
                              int32_t batch, float lr, uint64_t seed,
                              double* epoch_loss);
/* Searches of this context with params.seeded = 1 start each node's swarm
 * from prop: particle i at sigma (mu_hat + rho_i u_i / |u_i|) (as
 * slm_swarm_seed), mu_hat = o[0:d]/|o[0:d]|, rho_i = softplus(o[256 + i]);
 * requires d <= 256, n_classes <= 20 (or MSE),
 * n_particles <= 64. The context does not own prop; NULL detaches it. */
slm_status slm_use_proposal(slm_ctx* ctx, const slm_proposal* prop);
/* The seeded positions pos[P x d] for given mu_hat[d] and rho[P] (host or
 * device): x_ij = sigma (mu_hat_j + rho_i (u_ij / |u_i|)) in float, one
 * rounding per operation, u_ij = 2 U - 1 with U the swarm draw of purpose 6
 * at iteration 0 (slm_swarm_uniforms), |u_i| the correctly rounded square
 * root of a sequential fused multiply-add sum of squares and sigma =
 * sqrt(d / 3) rounded from d / 3 rounded (the expected norm of a uniform
 * start in [-1, 1)^d: seeded and random starts then have the same scale, and
 * the start velocities the same relative size). */
slm_status slm_swarm_seed(slm_ctx* ctx, uint64_t seed, uint32_t node_uid,
                          int32_t n_particles, int32_t d, const float* mu_hat,
                          const float* rho, float* pos);
/* The start a seeded search (params.seeded = 1, the context's proposal)
 * gives node (X rows sample_idx, labels / y, weights, node_uid; arguments as
 * slm_node_split): pos_out[n_particles x d] (host or device) receives the
 * positions of the node's initial swarm, computed by the search's own
 * kernels (node statistics, network forward, slm_swarm_seed's rule) as the
 * search would. SLM_EINVAL without a proposal in use or params.seeded != 1;
 * the seeded limits of slm_use_proposal apply. */
slm_status slm_seeded_start(slm_ctx* ctx, const slm_params* params, const float* X, int64_t n,
                            int32_t d, const int32_t* labels, const float* y,
                            const int32_t* sample_idx, const uint32_t* weights, int64_t n_idx,
                            uint32_t node_uid, float* pos_out);

/* ---- diagnostics --------------------------------------------------------
 * Kernels of this library, for per-kernel timing. */
typedef enum {
  SLM_K_PROJECT = 0,      /* z = X_node . x_p for every particle (FP32 FFMA) */
  SLM_K_HIST_SCAN = 1,    /* binning, histograms, threshold scan and, in a
                             search, the pbest / gbest steps of Algorithm 1 */
  SLM_K_SWARM_UPDATE = 2, /* Eq. pso-1 move of every particle */
  SLM_K_SWARM_INIT = 3,
  SLM_K_NODE_STATS = 4,
  SLM_K_PARTITION = 5,
  SLM_K_COMPACT = 6,
  SLM_K_GATHER = 7,       /* rows of a node / root into entry order */
  SLM_K_OTHER = 8,        /* validation, bootstrap, index setup, prediction */
  SLM_K_PROJECT_MMA = 9,  /* z in bfloat16 on the tensor cores (BF16_TOPK) */
  SLM_K_TOPK = 10,        /* BF16_TOPK: position conversion, top-k selection,
                             score merge with the pbest / gbest steps */
  SLM_K_PROPOSAL = 11,    /* node statistics, network passes, Adam, seeding */
  SLM_K_NODE_SEARCH = 12, /* whole searches of nodes held in shared memory */
  SLM_K_COUNT = 13
} slm_kernel;

/* on != 0 brackets every later launch of the context with CUDA events on its
 * stream; the counters restart at zero. Timing adds an event record per
 * launch and is meant for profiling runs. */
slm_status slm_profile(slm_ctx* ctx, int on);
/* Totals since slm_profile(ctx, 1) for one kernel: launches, summed event
 * time (ms; 0 while profiling is off) and particle-sample pairs the launches
 * scored (scoring kernels; 0 for the others). Synchronises the stream. */
slm_status slm_kernel_stats(slm_ctx* ctx, int32_t kernel, int64_t* launches,
                            double* total_ms, double* pairs);
/* Kernels launched by the context since its creation (a kernel run as a
 * node of a graph counts as one launch). */
slm_status slm_launch_count(slm_ctx* ctx, int64_t* launches);

/* Projection tiles. on = 1 (the default): the FP32 projection of a search
 * runs with the tile shape (particles per group: 8, 16, 24, 32 or 48 dividing
 * P rounded up to 16; 1 or 2 CTAs per SM; rows from the level copy or, in
 * bagged forests, gathered from the base rows) that was fastest when the first
 * search of the same shape (d, padded P, log2 of the 256-row tiles) timed
 * every candidate on its own batch; the choice is kept by the context. The
 * same first search also times the cluster histogram kernel with 1 to 16
 * CTAs per (node, particle) and keeps the fastest for the shape (criterion,
 * bins, classes, particles, multiplicities, log2 of the largest node and of
 * the node count). on = 0: 16 particles per group, 2 CTAs per SM, and the
 * largest power-of-two cluster that keeps the histogram grid in one wave.
 * Results are identical for every choice. SLM_EINVAL for other values. */
slm_status slm_set_tuning(slm_ctx* ctx, int32_t on);
/* Test hooks for the failure paths (no GPU fault is made):
 * first_wait_polls: polls of the histogram kernel's first wait on each
 * staged piece, for every context on ctx's device (< 0 restores the default
 * bound; 0 makes every wait give up at once: the kernel drains the copies in
 * flight, sets the error word and ends, and the call returns SLM_ETIMEOUT).
 * fail_alloc_after: the fail_alloc_after-th later growth of a library work
 * buffer fails as if the device were out of memory (SLM_ENOMEM; 0: never);
 * process-wide. Synchronises ctx's stream. SLM_EINVAL if
 * fail_alloc_after < 0. */
slm_status slm_test_hooks(slm_ctx* ctx, int32_t first_wait_polls, int64_t fail_alloc_after);

/* on = 1: a classification search (FP32 form) whose nodes'
 * rows, labels and multiplicities all fit in one SM's shared memory (about
 * n (d + 2) 4 bytes per node, with room for eight B x K histograms) runs all
 * of Algorithm 1's T + 1 iterations in one persistent launch: a cluster of
 * up to 8 CTAs per node, the node resident in each CTA's shared memory, one
 * warp per particle at a time. on = 0 (the default): the per-iteration
 * kernels, which measured as fast or faster on the workloads here. Scores,
 * trajectories and trees are identical either way. SLM_EINVAL for other
 * values. */
slm_status slm_set_node_search(slm_ctx* ctx, int32_t on);
/* CTAs per node of the context's last search in the persistent kernel, 0 if
 * the last search used the per-iteration kernels. */
slm_status slm_last_node_search(slm_ctx* ctx, int32_t* ctas_per_node);
/* Histogram kernels of classification searches (FP32 form): when a level's
 * nodes of at most max_entries entries (default 4096) give at least
 * min_pairs (node, particle) pairs (-1, the default: 2 x SMs x 8, enough
 * warps to fill the GPU), they are scored one warp per (node, particle)
 * from memory; the other nodes (all nodes otherwise) by clusters of CTAs
 * staging the node through shared memory. max_entries = 0 sends every node
 * to the clusters. Scores are identical either way. SLM_EINVAL for
 * max_entries < 0 or min_pairs < -1. */
slm_status slm_set_small_nodes(slm_ctx* ctx, int32_t max_entries, int64_t min_pairs);
/* Forces one tile shape for later searches (pg = 0 clears); gather = 1 reads
 * gathered base rows where a forest keeps them (elsewhere the level copy is
 * the only source). SLM_EINVAL for shapes outside the list above, and from a
 * search whose padded P pg does not divide. */
slm_status slm_force_tiles(slm_ctx* ctx, int32_t pg, int32_t ctas_per_sm, int32_t gather);
/* Shapes tuned so far, the tiles of the last search and the CTAs per
 * (node, particle) of its cluster histogram kernel (any may be NULL). */
slm_status slm_tuning_stats(slm_ctx* ctx, int64_t* shapes, int32_t* last_pg,
                            int32_t* last_ctas_per_sm, int32_t* last_hist_cluster);
/* The tuned shapes: *n receives their number; the first max are written to
 * the arrays (any may be NULL): features d, padded P, log2 of the row tiles,
 * the chosen particles per group, CTAs per SM and row source (1: gathered
 * from the base rows by sample id; the level's entry-ordered copy staged by
 * per-thread copies: 0, by tensor-map tile copies: 2), and
 * the chosen candidate's time for two projections (ms). Bagged forests whose
 * base rows fit in a quarter of L2 keep a copy of them, which makes the
 * gathered source a candidate for their levels. */
slm_status slm_tuned_shapes(slm_ctx* ctx, int32_t max, int32_t* n, int32_t* d,
                            int32_t* padded_p, int32_t* tiles_log2, int32_t* pg,
                            int32_t* ctas_per_sm, int32_t* gather, float* ms);

/* on = 1: the T + 1 scoring passes of every search (one node, or all nodes
 * of a level across all trees; Algorithm 1's loop) run as one CUDA graph
 * launch. The context keeps up to 64 executable graphs: a search
 * with exactly the launch inputs of a kept graph (sizes, parameters, tiles
 * and buffers) launches it again without recording; otherwise the passes are
 * recorded and a kept graph with the same launch shapes is updated in place,
 * or a new one is instantiated. on = 0 (the default): the passes are launched
 * one by one, chained by programmatic dependent launch.
 * Results are identical either way; per-launch profiling (slm_profile)
 * always launches one by one. SLM_EINVAL for other values. */
slm_status slm_set_graphs(slm_ctx* ctx, int32_t on);
/* on != 0 (the default): the FP32 projection stages rows that are contiguous
 * in memory (not gathered through sample ids), when d % 4 == 0 and the rows
 * are 16-byte aligned, by tensor-map tile copies (cp.async.bulk.tensor, one
 * issuing thread, 128-byte swizzle); on = 0: by per-thread asynchronous
 * copies. The projected values are identical either way. */
slm_status slm_set_projection_tma(slm_ctx* ctx, int32_t on);
/* on = 1 (the default) or 2: plain FP32 searches (no adaptive PSO, no BF16
 * form, no persistent node search) whose padded swarm is 16, 32, 48 or 64
 * particles, whose positions fit in 96 KB of shared memory and for which
 * no projection tiles are forced (slm_force_tiles) fold the
 * swarm move of Eq. pso-1 into the projection: one iteration is the
 * projection (which first takes the gbest step of the previous evaluation,
 * Algorithm 1, and moves every particle) and the histogram pass (which
 * leaves the gB-independent terms of the next move), two launches instead
 * of three, and each row tile is projected onto all particles at once.
 * With on = 1 only a batch whose projection is at most 4 waves of row
 * tiles (of 128 or 256 rows) on the GPU is folded: there the iteration is
 * latency-bound and the saved launch pays; longer projections (many nodes,
 * or one very large node) run faster unfolded, with the tuned projection.
 * on = 2 folds every eligible batch; on = 0 none (the projection,
 * histogram and move kernels). Results are identical either way.
 * *searches (optional) = searches run folded so far. SLM_EINVAL for other
 * values of on. */
slm_status slm_set_fused_step(slm_ctx* ctx, int32_t on, int64_t* searches);
/* Tile shape of the folded projection: shape = -1 (the default) picks, per
 * batch, the shape with the least estimated work per CTA (units per CTA x
 * (rows per unit x particles per unit / swarm width + a fixed cost of 32
 * rows per unit); on ties, half-swarm units where each CTA takes one unit,
 * else larger row tiles), so a short node is spread over
 * more CTAs; 0, 1, 2 force 128-256, 64-128 or 32-64 rows per tile with every
 * particle in a unit, 3, 4, 5 the same with half the particles of a swarm of
 * 32 or 64 (by swarm width; a width without the forced shape takes shape
 * 0). Results are identical for every shape. *last (optional) = the shape
 * of the last folded batch (-1 before the first). SLM_EINVAL for other
 * values of shape. */
slm_status slm_set_step_shape(slm_ctx* ctx, int32_t shape, int32_t* last);
/* on != 0 (the default): the searches of the FP32 form score each
 * iteration with the latency-oriented histogram kernels (entries loaded 16
 * bytes at a time with several in flight; classification: class-major
 * histograms scanned one warp per class; regression, for nodes of at most
 * 257,740 entries: two particles per block, the fixed-point bin moments
 * added as 32-bit pieces into lane copies; the pbest step spread over the
 * block; the BF16 form's regression passes too); on = 0: with
 * the staged-copy histogram kernel that also serves bins output and the
 * BF16 form. node_step != 0: in folded classification searches
 * (slm_set_fused_step) whose nodes all take that kernel, the last block to
 * score a node takes the node's gbest step (Algorithm 1) and moves its
 * particles (Eq. pso-1) once, instead of every projection block doing it;
 * node_step = 0 (the default): the projection blocks do it. Results are
 * identical in every combination. */
slm_status slm_set_class_hist(slm_ctx* ctx, int32_t on, int32_t node_step);
/* Roofline measurement (not part of the method): on `device`, with CUDA
 * events on `cuda_stream` (NULL = legacy default stream), *ffma_tflops
 * receives the FP32 fused multiply-add throughput of a kernel of independent
 * FMA chains filling every SM (2 flop per FMA; best of three timed launches
 * after a warm-up), the roof of the projection, whose rows stay in L2
 * across a search's iterations; *l2_read_gbs receives the read bandwidth of
 * a 48 MB L2-resident buffer streamed with 16-byte cache-global loads, the
 * roof of the histogram kernels, which read what the projection wrote.
 * Either pointer may be NULL (not both). The call allocates and frees its
 * own buffers, synchronises the stream, and restores the calling thread's
 * current device. Errors: SLM_EINVAL, SLM_ECUDA. */
slm_status slm_measure_peaks(int device, void* cuda_stream, double* ffma_tflops,
                             double* l2_read_gbs);
/* Graph launches of the context: in total, of kept graphs launched again
 * unchanged, updated in place, and instantiated anew (any may be NULL). */
slm_status slm_graph_stats(slm_ctx* ctx, int64_t* launches, int64_t* reuses,
                           int64_t* updates, int64_t* instantiations);

#ifdef __cplusplus
}
#endif
#endif
