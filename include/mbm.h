/*
 * mbm.h - C ABI of the GB300 Axilrod-Teller three-body engine.
 *
 * The library computes, for every particle x_i of a 3-D point set X,
 *
 *   Phi(x_i) = sum_{j<k; j,k != i} phi(x_i, x_j, x_k)                (Eq. 1, n = 3)
 *   phi(x_i,x_j,x_k) = (1 + 3 cos t_i cos t_j cos t_k)
 *                      / (r_ij^3 r_ik^3 r_jk^3)                       (Sec. 1, Axilrod-Teller)
 *
 * exactly (every unordered triple once, credited to its three members), or
 * approximately by the multi-tree method of Lee, Ozakin & Gray (Algorithm 2
 * with the p = 0 bounds of Sec. 4 and the Monte Carlo rules of
 * Algorithms 3-5), under the error criteria of Definitions 2.1-2.3.
 *
 * Conventions shared by every entry point:
 *   - X is N x 3 row-major FP64 (x0 y0 z0 x1 y1 z1 ...), caller-owned.
 *   - Outputs are caller-owned FP64 arrays. "_dev" pointers are device
 *     memory of the context's GPU; "_host" pointers are host memory.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and is asynchronous unless the entry point says otherwise.
 *     The caller must keep inputs and outputs alive until the stream has
 *     passed the call.
 *   - N < 3: the sum is empty, outputs are zeroed, MBM_OK (Eq. 1).
 *   - No exception crosses the ABI; every entry point returns a status and
 *     mbm_last_error() gives a thread-local message for the last failure.
 *   - The library owns its scratch memory (packed coordinates, work
 *     counters, trees); it is charged against the context's HBM budget.
 */
#ifndef MBM_H
#define MBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* mbm_stream_t; /* same handle as cudaStream_t */

typedef enum {
    MBM_OK = 0,
    MBM_PENDING = 1,     /* mbm_poll: request not finished yet */
    MBM_EINVAL = -1,     /* bad argument, non-finite or coincident points */
    MBM_ENOMEM = -2,     /* device allocation failed */
    MBM_EBUDGET = -3,    /* request does not fit the context's HBM budget */
    MBM_EOVERFLOW = -4,  /* a bounded device work list overflowed */
    MBM_ETIMEDOUT = -5,  /* a bounded wait ran out */
    MBM_ECUDA = -6,      /* a CUDA runtime call failed */
    MBM_ENOTSUP = -7     /* mode not supported by this entry point */
} mbm_status;

/* Modes of mbm_potential / mbm_forces. */
enum {
    MBM_EXH_FP64 = 0, /* exhaustive, FP64 everywhere */
    MBM_EXH_FP32 = 1, /* exhaustive, FP32 triple arithmetic, FP64 accumulation */
    MBM_TREE = 2,     /* multi-tree approximation (Algorithm 2) */
    MBM_ABS = 0x100   /* with MBM_TREE: eps is the absolute bound tau (Def. 2.1) */
};

/* Tuning and semantics of the tree path (Sec. 3-4). */
typedef struct {
    double tau;          /* absolute error term of Def. 2.3 (0 = pure relative) */
    int32_t leaf_size;   /* leaf threshold of Algorithm 1 (default 32, range 2..32) */
    int32_t m_limit;     /* Monte Carlo sample cap of Algorithm 4 (default 256, <= 65535) */
    double zeta;         /* speed-up factor of Algorithm 3 (default 32) */
    uint64_t seed;       /* Philox-4x32-10 key for Monte Carlo draws */
    int32_t mc_rule;     /* 0 = relative stop test with T_i on both terms, 1 = as printed */
    int32_t validate;    /* 1: synchronise and report non-finite/coincident input */
    int32_t seed_levels; /* Phi^l seed node = ancestor this many levels above a leaf, 0-8
                            (default 8); the force criterion's A^l seed uses at most 6 */
    int32_t reserved0;
    int64_t* tuple_counts; /* optional device int64[N]: point triples credited to each
                              particle by prunes and base cases (validation; NULL = off) */
    /* Traversal buffer sizes, 0 = sized from N (the default). Smaller values
     * change only how the work is batched, never a decision or a result:
     * they exist so that small test problems run the paths large ones take. */
    int32_t trav_chunk;    /* node triples classified per launch (>= 1) */
    int32_t base_cap;      /* leaf triples per base-case flush (raised to >= trav_chunk) */
    int32_t est_cap;       /* Monte Carlo estimates per batch (raised to >= N + 128) */
    int32_t reserved1;
} mbm_config;

/* Counters of the last solve (tree path); all zero for exhaustive modes. */
typedef struct {
    int64_t node_triples_visited;
    int64_t det_prunes;
    int64_t mc_prunes;
    int64_t mc_attempts;
    int64_t base_cases;
    int64_t base_triples;   /* point triples evaluated exactly */
    int64_t mc_samples;     /* phi evaluations drawn by Monte Carlo */
    int64_t levels;         /* traversal levels */
    double ms_build, ms_seed, ms_traverse, ms_base, ms_finalize;
    int64_t chunks;         /* classify launches */
    int64_t base_flushes;   /* base-case flushes */
    int64_t mc_batches;     /* Monte Carlo estimate batches */
} mbm_stats;

typedef struct mbm_ctx mbm_ctx;
typedef struct mbm_tree mbm_tree;

/* Version string of the library. */
const char* mbm_version(void);

/* Message for the last failing call on this thread ("" if none). */
const char* mbm_last_error(void);

/* Fill *cfg with the defaults listed above. */
void mbm_config_default(mbm_config* cfg);

/* Create a context on CUDA device `device` whose library-owned device
 * memory may not exceed `hbm_budget_bytes` (0 = no limit). *out is
 * owned by the caller and released with mbm_ctx_destroy. */
mbm_status mbm_ctx_create(int device, size_t hbm_budget_bytes, mbm_ctx** out);

/* Synchronise the device and free every library-owned buffer. */
mbm_status mbm_ctx_destroy(mbm_ctx* ctx);

/* Library-owned device bytes currently held by the context. */
size_t mbm_ctx_bytes_in_use(const mbm_ctx* ctx);

/* Enable (1) or disable (0) CUDA-event timing of each solve's dominant
 * kernel (the exhaustive kernel, or the tree path's base-case kernels).
 * Events are recorded on the solve's stream. */
mbm_status mbm_ctx_set_timing(mbm_ctx* ctx, int enable);

/* Milliseconds spent in the dominant kernel(s) of the last timed solve;
 * waits for that solve's end event. Returns -1 if nothing was timed. */
double mbm_ctx_last_kernel_ms(mbm_ctx* ctx);

/*
 * Phi(x_i) for all i (Eq. 1 with the Axilrod-Teller phi of Sec. 1).
 *   X_dev   : N x 3 FP64 device array, read only.
 *   phi_dev : N FP64 device array, written (fully overwritten).
 *   mode    : MBM_EXH_FP64, MBM_EXH_FP32, or MBM_TREE[|MBM_ABS].
 *   eps     : tree modes only; relative bound of Def. 2.2 (or tau with
 *             MBM_ABS, Def. 2.1). Must be >= 0.
 *   alpha   : tree modes only; failure probability of Def. 2.3, in [0, 1).
 *             alpha = 0 selects the deterministic rule.
 * Errors: MBM_EINVAL for N < 0, NULL pointers, eps < 0, alpha outside
 * [0, 1), an unknown mode; with cfg->validate (default on in
 * mbm_potential) also for non-finite coordinates or two coincident points,
 * detected on the device and reported after a stream synchronisation.
 */
mbm_status mbm_potential(mbm_ctx* ctx, const double* X_dev, int64_t N, double eps,
                         double alpha, int mode, double* phi_dev, mbm_stream_t stream);

/* As mbm_potential, with explicit configuration (NULL = defaults), an
 * optional prebuilt tree for MBM_TREE (NULL = build one internally) and an
 * optional stats record (NULL = not reported; filling it synchronises). */
mbm_status mbm_potential_ex(mbm_ctx* ctx, const double* X_dev, int64_t N, double eps,
                            double alpha, int mode, const mbm_config* cfg, mbm_tree* tree,
                            double* phi_dev, mbm_stats* stats, mbm_stream_t stream);

/* Host-buffer variant: copies X_host to the device, runs mbm_potential_ex
 * and copies Phi back to phi_host, then synchronises `stream`.
 * Device buffers are library-owned scratch. */
mbm_status mbm_potential_host(mbm_ctx* ctx, const double* X_host, int64_t N, double eps,
                              double alpha, int mode, const mbm_config* cfg,
                              double* phi_host, mbm_stream_t stream);

/*
 * Exact Phi (Eq. 1) of selected particles only, FP32 bulk with FP64
 * accumulation: out_dev[q] = Phi(x_{idx_dev[q]}) over all pairs j < k of the
 * whole set. Used as the reference for tree accuracy at sizes where the full
 * exhaustive sum is out of reach (cost: n_idx * C(N-1, 2) triples).
 *   idx_dev : n_idx int64 device indices in [0, N) (0 <= n_idx <= 2^20).
 *   out_dev : n_idx FP64 device array, written.
 * Indices outside [0, N) are skipped on the device (their output stays 0)
 * and reported as MBM_EINVAL; non-finite coordinates likewise. Synchronises
 * `stream` once at the end to read those flags.
 */
mbm_status mbm_potential_sampled(mbm_ctx* ctx, const double* X_dev, int64_t N,
                                 const int64_t* idx_dev, int64_t n_idx, double* out_dev,
                                 mbm_stream_t stream);

/*
 * Three-body far-field expansion (Sec. 3.2, Eq.
 * truncated_three_body_farfield_expansion) of Axilrod-Teller sums: for each
 * query point x (Xq_dev, nq x 3 FP64, device) the p-th order expansion of
 *
 *   Phi(x; P2 x P3) = sum_{y2 in P2} sum_{y3 in P3} phi(x, y2, y3)
 *
 * about the centres of mass c2, c3 of the source sets P2 (Y2_dev, n2 x 3) and
 * P3 (Y3_dev, n3 x 3), with the far-field moments of Sec. 3.1 up to order p.
 * Axilrod-Teller enters as ten products of pairwise powers (law of cosines).
 * p = 0 is the monopole n2 n3 phi(x, c2, c3) of the p = 0 rule (Sec. 4); the
 * error falls with p where the query and source sets are well separated
 * (|y - c| small against the distances between x, c2 and c3).
 *   out_dev: caller-owned FP64[nq] on the device.
 *   p: 0..6. Moments and the source-dependent coefficients are FP64; each
 *   query point is evaluated in FP32 arithmetic from FP64 differences x - c.
 *   n2 == 0 or n3 == 0: the double sum is empty, out = 0.
 *   The sets are taken as given: the caller keeps x out of P2 and P3 (as for
 *   distinct tree nodes); P2 and P3 may share points, but not a centre.
 *   validate = 1 synchronises `stream` and reports a non-finite coordinate
 *   or a query point at a centre, or c2 == c3 (the expansion is undefined
 *   there), as MBM_EINVAL; with validate = 0 such outputs are NaN or Inf.
 * Errors: MBM_EINVAL (bad p, NULL pointer, negative size), MBM_EBUDGET,
 * MBM_ENOMEM. Scratch: a few hundred KB from the context's arena.
 */
mbm_status mbm_farfield3(mbm_ctx* ctx, const double* Xq_dev, int64_t nq, const double* Y2_dev,
                         int64_t n2, const double* Y3_dev, int64_t n3, int p, int validate,
                         double* out_dev, mbm_stream_t stream);

/*
 * Build the spatial tree of Sec. 3 (bottom-up phase) for X_dev (N x 3 FP64,
 * device): Morton-ordered permutation, balanced node ranges of at most
 * cfg->leaf_size points, FP64 bounding boxes and centres of mass, and the
 * Phi^l seed of every node. The tree copies what it needs from X_dev and is
 * owned by the caller (mbm_tree_free). Asynchronous on `stream` except for
 * one size read-back. Errors: MBM_EINVAL (N < 3, bad leaf_size), MBM_EBUDGET,
 * MBM_ENOMEM.
 */
mbm_status mbm_tree_build(mbm_ctx* ctx, const double* X_dev, int64_t N, const mbm_config* cfg,
                          mbm_stream_t stream, mbm_tree** out);

/* Release a tree (synchronises its device). */
mbm_status mbm_tree_free(mbm_tree* tree);

/* Number of nodes and leaves of a tree (for inspection). */
mbm_status mbm_tree_info(const mbm_tree* tree, int64_t* n_nodes, int64_t* n_leaves,
                         int32_t* depth);

/* Copy a tree's layout to caller-owned device arrays (any may be NULL):
 * perm_dev (int64[N], sorted position -> original index), lo_dev/hi_dev
 * (FP64[3 * n_nodes], boxes), cen_dev (FP64[3 * n_nodes], centres of mass),
 * phil_dev (FP64[n_nodes], Phi^l seed). Nodes are in heap order (root 0,
 * children 2v+1, 2v+2). Asynchronous on `stream`. */
mbm_status mbm_tree_export(const mbm_tree* tree, int64_t* perm_dev, double* lo_dev,
                           double* hi_dev, double* cen_dev, double* phil_dev,
                           mbm_stream_t stream);

/*
 * Forces F_i = -dE/dx_i of the total energy E = sum_{a<b<c} phi_abc
 * (no counterpart in the paper; the derivative of Eq. 1's summand).
 *   F_dev : N x 3 FP64 device array, written.
 *   mode  : MBM_EXH_FP64 or MBM_EXH_FP32 (exhaustive adjoint), or MBM_TREE[|MBM_ABS]:
 *           the multi-tree recursion (Algorithm 2's traversal and splits)
 *           under a force criterion, since the paper bounds potentials only:
 *           every component of F_i within eps S_i + tau, where
 *           S_i = sum over the tuples containing i of |grad_i phi|_2 (a sum of
 *           magnitudes, which cancelling terms cannot shrink); MBM_ABS makes
 *           eps the absolute tau. A pruned node triple credits
 *           -T_s grad_s phi(c1, c2, c3) (p = 0: pruned when 2 M_s <=
 *           (eps A^l + tau)/T^root with M_s a bound on |grad phi| over the
 *           boxes and A^l <= S the exact sum over the seed node) or, with
 *           alpha > 0, a Monte Carlo mean (Algorithms 3-5 with the three
 *           components as the sample); base cases are exact.
 */
mbm_status mbm_forces(mbm_ctx* ctx, const double* X_dev, int64_t N, double eps, double alpha,
                      int mode, double* F_dev, mbm_stream_t stream);

/* As mbm_forces, with explicit configuration (NULL = defaults), an optional
 * prebuilt tree for MBM_TREE (NULL = build one) and an optional stats record
 * (NULL = not reported; filling it synchronises). */
mbm_status mbm_forces_ex(mbm_ctx* ctx, const double* X_dev, int64_t N, double eps, double alpha,
                         int mode, const mbm_config* cfg, mbm_tree* tree, double* F_dev,
                         mbm_stats* stats, mbm_stream_t stream);

/*
 * Vector-Jacobian product of Phi: gradX_m = d/dx_m sum_l g_l Phi(x_l)
 * = sum over triples t containing m of (g_a + g_b + g_c) d phi_t/d x_m.
 *   g_dev     : N FP64 device array (cotangent of Phi).
 *   gradX_dev : N x 3 FP64 device array, written.
 *   mode      : MBM_EXH_FP64 or MBM_EXH_FP32.
 */
mbm_status mbm_potential_vjp(mbm_ctx* ctx, const double* X_dev, int64_t N, const double* g_dev,
                             int mode, double* gradX_dev, mbm_stream_t stream);

/*
 * Exhaustive FP32-bulk Phi (as mbm_potential with MBM_EXH_FP32) for callers
 * that cannot let a library allocate device memory: applications that own
 * every device byte through their own pool or budget, loops that cannot
 * afford the synchronisation an allocation or free brings, or plugins in a
 * process that forbids foreign allocations. The paper has no counterpart;
 * this is a deployment variant of the exhaustive sum.
 *   X_dev   : N x 3 FP64 device array (current device), read only.
 *   phi_dev : N FP64 device array, written.
 *   N       : 0 <= N <= 65536; larger N returns MBM_EINVAL (use mbm_potential).
 * No device memory is allocated or freed: scratch is a fixed 2 MiB + 256 B
 * file-scope device array that every GPU loading the library holds until
 * exit. The first call on a device resolves that array's device address
 * (cudaGetSymbolAddress) and caches it for the rest of the process; make
 * that first call before any stream capture. The cached address belongs to
 * the device's primary context: after cudaDeviceReset (or with another
 * context current) it is stale, so such callers must not use this entry
 * point again in the same process. Every call shares the one array, so calls whose work
 * overlaps on the GPU (different streams, or concurrent host threads) race;
 * serialise them. No input validation on the device: non-finite or
 * coincident points give non-finite results rather than MBM_EINVAL.
 */
mbm_status mbm_potential_fp32_noalloc(const double* X_dev, int64_t N, double* phi_dev,
                                      mbm_stream_t stream);

/* ------------------------------------------------------------------------
 * Serving (no counterpart in the paper): continuous batching of potential
 * and force requests of uneven N on one GPU. Each of `slots` workers owns a
 * context and a non-blocking stream; a request starts as soon as a slot is
 * free and its estimated device footprint fits the budget (oldest first, with
 * backfill of younger requests that fit beside the room held for the oldest),
 * so requests overlap on the device. A non-zero system_id keeps that point
 * set (and its tree, for tree solves) resident until evicted (least recently
 * used, when the budget needs the room); a system id names a fixed point set.
 * ------------------------------------------------------------------------ */
typedef struct mbm_server mbm_server;

enum { MBM_REQ_POTENTIAL = 0, MBM_REQ_FORCES = 1 };

typedef struct {
    int32_t kind;          /* MBM_REQ_POTENTIAL or MBM_REQ_FORCES */
    int32_t mode;          /* MBM_EXH_FP32 / MBM_EXH_FP64 / MBM_TREE[|MBM_ABS] (both kinds) */
    int64_t N;
    const double* X_host;  /* N x 3 FP64, caller-owned, read while the request runs */
    double* out_host;      /* N (potential) or N x 3 (forces) FP64, caller-owned, written */
    double eps, alpha;     /* tree modes (as in mbm_potential) */
    uint64_t system_id;    /* != 0: keep / reuse this point set on the device */
    const mbm_config* cfg; /* NULL = defaults; copied by mbm_submit */
} mbm_request;

typedef struct {
    int32_t status;        /* status of the solve */
    int32_t slot;          /* worker that ran it */
    double queue_ms;       /* submit -> start */
    double compute_ms;     /* start -> result in out_host */
    double latency_ms;     /* submit -> result in out_host */
    int64_t bytes_reserved;/* footprint estimate admitted against the budget */
    int64_t dev_start_ns;  /* device clock (%globaltimer, ns) when the solve's first kernel */
    int64_t dev_end_ns;    /* started / after its last kernel; intervals of requests that
                              ran at once overlap (0 if the request failed) */
} mbm_result;

/* Create a server on `device` with `slots` (1..64) workers and an HBM budget
 * (0 = none). Buffers and contexts are owned by the server. */
mbm_status mbm_server_create(int device, size_t hbm_budget_bytes, int32_t slots,
                             mbm_server** out);

/* Stop the workers (requests not yet started are dropped) and free everything. */
mbm_status mbm_server_destroy(mbm_server* server);

/* Queue a request; *ticket identifies it. The request struct is copied; the
 * caller keeps X_host and out_host alive until mbm_poll reports completion.
 * MBM_EBUDGET if its estimated footprint alone exceeds the budget. */
mbm_status mbm_submit(mbm_server* server, const mbm_request* req, uint64_t* ticket);

/* Wait up to timeout_us (0 = do not wait, < 0 = forever) for a ticket.
 * Returns MBM_OK with *res filled (res->status is the solve's status),
 * MBM_PENDING (timeout_us = 0, not finished), MBM_ETIMEDOUT, or MBM_EINVAL
 * for an unknown or already collected ticket. */
mbm_status mbm_poll(mbm_server* server, uint64_t ticket, mbm_result* res, int64_t timeout_us);

/* Counters: requests admitted, waiting, rejected, completed; bytes held. */
mbm_status mbm_server_stats(mbm_server* server, int64_t* admitted, int64_t* pending,
                            int64_t* rejected, int64_t* completed, size_t* reserved);

#ifdef __cplusplus
}
#endif
#endif /* MBM_H */
