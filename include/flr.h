/*
 * flr.h -- C ABI of the GB300 fused lasso regression (FLR) solver.
 *
 * Problem (Section 1, Eq. obj):
 *     minimise  f(beta) = 1/2 ||y - X beta||^2 + lambda1 sum_j |beta_j|
 *                         + lambda2 sum_{(j,k) in E} |beta_j - beta_k|
 * solved by the majorization-minimization (MM) iteration of Section 3:
 * each MM iteration r reweights a_j = 1/(|beta_j| + eps) and
 * w_jk = 1/(|beta_j - beta_k| + eps) from the current iterate and solves the
 * symmetric positive-definite surrogate system (Eq. lin-sys)
 *     (X^T X + lambda1 A(r) + lambda2 B(r)) beta = X^T y
 * by preconditioned conjugate gradient warm-started at beta(r)
 * (Algorithm 2), until the relative change of f is at most tol
 * (Algorithm 1/2 outer stop).  The limit minimises the perturbed objective
 * f_eps of Eq. pert.
 *
 * Conventions for every entry point:
 *   - Return values are flr_status codes; nothing is thrown across the ABI
 *     and nothing aborts.  flr_strerror() names a code.
 *   - "device" pointers are CUDA global-memory pointers on the current
 *     device; "host" pointers are ordinary (preferably pinned) host memory.
 *   - A handle is bound to the CUDA device that was current at flr_create
 *     and to the stream given there.  All work of a handle is issued on
 *     that stream.  A handle is not thread-safe; distinct handles are
 *     independent.
 *   - All reals are IEEE double unless the storage dtype of X says
 *     otherwise.
 */
#ifndef FLR_H
#define FLR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum flr_status {
    FLR_OK = 0,
    FLR_EINVAL = 1,       /* invalid argument (sizes, pointers, edge set, lambdas, eps, tol) */
    FLR_ENOMEM = 2,       /* a device or pinned-host allocation failed */
    FLR_ECUDA = 3,        /* a CUDA runtime call failed (launch, copy, device query) */
    FLR_ENOTCONV = 4,     /* max_mm MM iterations reached before the outer stop test held */
    FLR_EBREAKDOWN = 5,   /* CG met p^T Q p <= 0 (Q not SPD, e.g. lambda1 = 0 with singular X^T X + lambda2 B) */
    FLR_ENONFINITE = 6,   /* a non-finite value appeared (inputs or arithmetic) */
    FLR_ETIMEOUT = 7,     /* a bounded device-side wait gave up; results are not valid */
    FLR_ENOTIMPL = 8,     /* the requested combination is not implemented */
    FLR_ESCRATCH = 9      /* flr_solve_noalloc: the problem does not fit its static scratch */
} flr_status;

/* Storage type of X.  Products with X accumulate in FP32 for F32/BF16/F16
 * and in FP64 for F64; every other quantity is FP64.
 * FLR_IDENTITY: X = I with n = p, the fused lasso signal approximator (FLSA,
 * the special case of Eq. obj named in Section 1; Section 5.2 denoises an
 * image with it).  No matrix is passed (X = NULL, ldx ignored) and the solve
 * reads none: every X product is the vector itself, so each CG iteration is
 * the Laplacian stencil or CSR product and vector work only.  flr_create,
 * flr_solve and flr_solve_batch (one solve per pair) accept it; the server
 * and flr_solve_noalloc do not (FLR_EINVAL). */
typedef enum flr_dtype { FLR_F64 = 0, FLR_F32 = 1, FLR_BF16 = 2, FLR_F16 = 3, FLR_IDENTITY = 4 } flr_dtype;

/* Where the pointers passed to flr_create / flr_solve live. */
typedef enum flr_mem { FLR_MEM_DEVICE = 0, FLR_MEM_HOST = 1 } flr_mem;

/* The edge set E (Section 1).
 *   FLR_E_CHAIN:   E = {(j-1, j) : j = 1..p-1}, the standard FLR.  q1, q2,
 *                  edges, m are ignored.
 *   FLR_E_LATTICE: the two-dimensional FLR on a q1 x q2 lattice; coefficient
 *                  (i, j) has index i*q2 + j (row-major) and E holds the
 *                  horizontal and vertical neighbour pairs.  q1*q2 must equal p.
 *   FLR_E_EDGES:   an explicit list: `edges` holds m pairs (j, k) as 2*m
 *                  int64 values, 0-based, j != k, no pair listed twice in
 *                  either orientation (E is a set).  m = 0 is allowed. */
typedef enum flr_graph_kind { FLR_E_CHAIN = 0, FLR_E_LATTICE = 1, FLR_E_EDGES = 2 } flr_graph_kind;

typedef struct flr_graph {
    int32_t kind;           /* flr_graph_kind */
    int32_t reserved;
    int64_t q1, q2;         /* lattice shape */
    const int64_t* edges;   /* FLR_E_EDGES: 2*m values, in the memory named by flr_create's `mem` */
    int64_t m;
} flr_graph;

/* Preconditioner M of the inner PCG (Algorithm 2).  The preconditioner
 * changes the number of CG iterations, not the MM iterates' limit.
 *   FLR_PC_JACOBI:  M = diag(X^T X + lambda1 A + lambda2 B).
 *   FLR_PC_TRIDIAG: M = the tridiagonal part of X^T X + lambda1 A + lambda2 B
 *                   over consecutive indices, with diag(X^T X) in place of
 *                   X^T X; solved exactly within each block of consecutive
 *                   indices owned by one thread block (blocks decouple at
 *                   their ends).  On a chain this is the paper's tridiagonal
 *                   preconditioner plus diag(X^T X); on a lattice it is a
 *                   horizontal-line preconditioner.
 *   FLR_PC_PAPER:   as TRIDIAG but without diag(X^T X): M = lambda1 A + lambda2 B
 *                   restricted to consecutive-index couplings (Algorithm 2).
 *   FLR_PC_TWOLEVEL: a local part plus a coarse correction on the fused groups:
 *                   M^-1 r = L^-1 r + sum_c 1_c (1_c^T r) / q_c, with L the
 *                   TRIDIAG matrix on a chain and the diagonal of Q on other
 *                   graphs, c running over the connected components
 *                   (two or more coefficients) of the edges whose weight
 *                   lambda2 w_jk is at least 16 min(d_j + lambda1 a_j,
 *                   d_k + lambda1 a_k), 1_c their indicator vectors and q_c =
 *                   sum_{j in c}(d_j + lambda1 a_j) + the lambda2 w of the
 *                   edges leaving c.  Recomputed every MM iteration.  Any
 *                   graph kind.
 *   FLR_PC_AUTO:    TWOLEVEL (flr_solve_batch: its per-tile TRIDIAG). */
typedef enum flr_precond {
    FLR_PC_AUTO = 0, FLR_PC_JACOBI = 1, FLR_PC_TRIDIAG = 2, FLR_PC_PAPER = 3, FLR_PC_TWOLEVEL = 4
} flr_precond;

typedef struct flr_opts {
    int32_t max_mm;      /* MM iteration cap (default 10000, Section 5) */
    int32_t max_cg;      /* CG iterations per MM iteration (default 10000) */
    int32_t min_cg;      /* at least this many CG iterations per MM iteration (default 1) */
    int32_t precond;     /* flr_precond (default FLR_PC_AUTO) */
    double tol_cg;       /* inner stop ||r_j|| / ||X^T y|| <= tol_cg (default: tol, as Algorithm 2) */
    int32_t grid;        /* thread blocks of the solve kernel; 0 = automatic */
    int32_t inject_stall;/* test hook: 1 = block 0 leaves before the first grid barrier, so
                            the other blocks' bounded waits expire and the solve returns
                            FLR_ETIMEOUT (needs grid >= 2).  0 in normal use. */
    int64_t wait_cycles; /* bound of every device-side wait in SM clock cycles (0 = 2^33) */
    int32_t max_refine;  /* refinement restarts of the inner solve per MM iteration (default 0).
                            Every MM iteration starts CG from the residual c - Q x computed in
                            FP64.  With max_refine = R > 0, once CG meets tol_cg on its
                            recursive residual, the true residual of the same surrogate
                            system is recomputed in FP64 and CG restarts from it, at most R
                            times, until the true residual meets tol_cg too.  This solves
                            each surrogate to FP64 accuracy from FP32/BF16/FP16 products, so
                            the iterates follow the MM map of Algorithm 1 (mixed-precision
                            iterative refinement).  flr_solve_batch applies it per RHS. */
    int32_t x_smem;      /* where the X products read X (flr_solve; flr_solve_noalloc takes 0
                            or -1).  0 (default): the leading columns of each thread block's
                            slab stay on chip for the whole solve, in tensor memory (TMEM,
                            32- and 16-bit X, n <= 2048) and then in shared memory; the
                            rest are streamed, twice per CG iteration (X p, then X^T u).
                            -1: every column streamed twice per CG iteration.  1: the
                            one-pass Q-apply (32- and 16-bit X): each CG iteration reads X
                            once from memory in row chunks that stay in L2 between the X p
                            and X^T u halves of the product, with a grid-wide split barrier
                            per chunk; on GB300 it is slower than two passes at every
                            measured size, so it is never chosen by default. */
    double tol_cg_rel;   /* adaptive inner tolerance (default 0 = off; flr_solve,
                            flr_solve_noalloc and, per RHS, flr_solve_batch).  With theta = tol_cg_rel > 0, the inner solve
                            of MM iteration r stops when ||r|| / ||X^T y|| <= max(tol_cg,
                            min(theta * rel_r, ||r0|| / (2 ||X^T y||))), rel_r the relative
                            change of f that iteration's outer test just measured (1 at r = 0)
                            and r0 the solve's start residual: early surrogates, whose
                            solutions are far from the limit, are solved loosely, later ones
                            to tol_cg, and every solve at least halves its start residual.
                            Every CG iteration lowers the surrogate g_eps from its warm start,
                            so f_eps still decreases monotonically (Prop. 1, Lemma 2); the
                            fixed point is unchanged. */
} flr_opts;

typedef struct flr_stats {
    int32_t mm_iters;        /* MM iterations performed */
    int32_t cg_iters;        /* CG iterations summed over all MM iterations */
    int32_t status;          /* flr_status of the solve */
    int32_t grid;            /* thread blocks used */
    double f;                /* f(beta) at the returned beta (Eq. obj); the objective */
    double f_eps;            /* f_eps(beta) (Eq. pert) */
    double rel_change;       /* last |f(b_new) - f(b_old)| / |f(b_old)| */
    double cg_relres;        /* ||r|| / ||X^T y|| at the end of the last inner solve (the
                                FP64 true residual when the solve ended on a refinement) */
    double ms;               /* device time of the solve kernel, milliseconds */
    int32_t refine_steps;    /* FP64 refinement passes inside MM iterations (opts.max_refine) */
    int32_t reserved;
    double est_err;          /* estimated relative error of f against the exact minimum f* of
                                Eq. obj:  (f - f_eps)/f, the bound of Prop. 1(ii) on what the
                                perturbation costs, plus the MM tail rel_change * q / (1 - q)
                                with q = rel_change / (the change before it) capped at 0.999
                                (a linear-convergence estimate; rel_change alone when fewer
                                than two changes exist).  An estimate, not a bound. */
} flr_stats;

typedef struct flr_handle flr_handle;
typedef flr_handle* flr_t;

/* Fill *opts with the defaults listed in flr_opts. */
void flr_default_opts(flr_opts* opts);

/* Create a problem handle.
 *   X      n x p design matrix, row-major, row stride ldx >= p elements,
 *          element type `dtype` (FLR_BF16 / FLR_F16: 16-bit patterns);
 *          NULL with dtype FLR_IDENTITY (then n must equal p).
 *   y      n responses (double).
 *   E      edge set (see flr_graph); E->edges in the memory named by `mem`.
 *   mem    FLR_MEM_DEVICE or FLR_MEM_HOST: where X, y and E->edges live.
 *   stream cudaStream_t (NULL = legacy default stream).
 * The handle copies what it needs (X into a column-major layout of the
 * same dtype, y, the edge set) and computes X^T y and diag(X^T X) in FP64;
 * the caller's buffers may be released once this call returns.
 * Errors: FLR_EINVAL for n < 1, p < 1, ldx < p, a null pointer, an
 * unknown dtype or kind, q1*q2 != p, an edge index outside [0, p), a self
 * loop or a repeated pair; FLR_ENOMEM / FLR_ECUDA as named. */
flr_status flr_create(const void* X, int32_t dtype, int64_t n, int64_t p, int64_t ldx,
                      const double* y, const flr_graph* E, int32_t mem, void* stream,
                      flr_t* out);

/* Run the MM iteration for one (lambda1, lambda2).
 *   eps        perturbation constant of Eq. pert (> 0).
 *   tol        outer stop: |f(b(r+1)) - f(b(r))| / |f(b(r))| <= tol (> 0).
 *   opts       NULL for defaults.
 *   beta_init  NULL: beta(0)_j = X_j^T y / X_j^T X_j (0 for a zero column;
 *              Algorithm 1); else p doubles in `io_mem` memory.
 *   beta_out   p doubles in `io_mem` memory (may equal beta_init).
 *   io_mem     FLR_MEM_DEVICE or FLR_MEM_HOST for beta_init and beta_out.
 *   stats      optional (NULL allowed), host memory.
 * lambda1 = 0 is accepted; the surrogate system is then SPD only when
 * X^T X + lambda2 B is, otherwise FLR_EBREAKDOWN.  Returns FLR_ENOTCONV
 * (with beta_out written) when max_mm is reached.  The call returns after
 * the solve has finished on the handle's stream. */
flr_status flr_solve(flr_t h, double lambda1, double lambda2, double eps, double tol,
                     const flr_opts* opts, const double* beta_init, double* beta_out,
                     int32_t io_mem, flr_stats* stats);

/* Solve K independent (lambda1[k], lambda2[k]) problems on the same X, y, E
 * (a lambda grid).  betas is p x K column-major (column k = beta for pair k)
 * in `io_mem` memory; objectives (K doubles) and stats (K entries) are host
 * memory and optional.  Returns the first non-OK status over k, else FLR_OK.
 * BF16 X on a chain or lattice with precond AUTO, JACOBI, TRIDIAG or PAPER
 * runs one tensor-core launch per 64 pairs (AUTO: the per-tile tridiagonal
 * preconditioner); any other case solves the pairs one after another with
 * flr_solve.  The first tensor-core batch on a handle also tunes the launch:
 * it times one capped launch (one MM iteration, 24 CG iterations) for each of
 * up to three split-K chunk lengths of the X P contraction and keeps the
 * fastest for the handle's later batches. */
flr_status flr_solve_batch(flr_t h, int32_t K, const double* lambda1, const double* lambda2,
                           double eps, double tol, const flr_opts* opts, double* betas,
                           int32_t io_mem, double* objectives, flr_stats* stats);

/* Largest p flr_solve_dense accepts (its two p x p FP64 matrices take 16 p^2 bytes). */
#define FLR_DENSE_MAX_P 32768

/* Algorithm 1 as the paper states it: the same MM iteration as flr_solve, but
 * each surrogate system (Eq. lin-sys) is solved by a dense Cholesky
 * factorization, which the paper recommends for a general edge set (Section 4)
 * where CG may need many iterations.  Everything is FP64: G = X^T X is formed
 * once per handle (X widened exactly from its storage type) and kept; each MM
 * iteration forms Q = G + lambda1 A + lambda2 B, factors Q = L L^T by a blocked
 * right-looking Cholesky in 64 x 64 tiles, solves L L^T beta = X^T y, and
 * evaluates f(beta) from X beta.  The stop test is the relative change of f
 * (tol), at most max_mm MM iterations.  beta_init, beta_out, io_mem and stats as
 * in flr_solve (stats: cg_iters = 0, grid = 0, ms = host wall time).  The first
 * call allocates 16 p^2 bytes on the handle's device, released by flr_destroy.
 * Errors: FLR_EINVAL for invalid arguments; FLR_ENOTIMPL for FLR_IDENTITY X or
 * p > FLR_DENSE_MAX_P; FLR_EBREAKDOWN when a pivot is not positive (Q not SPD,
 * e.g. lambda1 = 0 with singular X^T X + lambda2 B); FLR_ENOTCONV at max_mm;
 * FLR_ENOMEM / FLR_ECUDA. */
flr_status flr_solve_dense(flr_t h, double lambda1, double lambda2, double eps, double tol,
                           int32_t max_mm, const double* beta_init, double* beta_out,
                           int32_t io_mem, flr_stats* stats);

/* Release a handle and everything it owns (NULL is ignored). */
void flr_destroy(flr_t h);

/* Static, NUL-terminated name and description of a status code. */
const char* flr_strerror(int32_t status);

/* Problem sizes of a handle (any out-pointer may be NULL). */
flr_status flr_get_info(flr_t h, int64_t* n, int64_t* p, int64_t* m, int32_t* dtype);

/* Bytes of the static device scratch array used by flr_solve_noalloc. */
#define FLR_NOALLOC_SCRATCH_BYTES (16u << 20)

/* The same MM solve as flr_solve, for callers that cannot allocate device
 * memory: it calls no cudaMalloc/cudaFree and no allocating library routine.
 * (The paper has no counterpart; this is a deployment entry point.)  Typical
 * such callers run inside a framework whose caching allocator has already
 * reserved the GPU's memory, so a new cudaMalloc would fail or fragment that
 * pool, or in a serving loop that must not take the driver's allocation
 * path, which can synchronize the device.
 *
 * All working memory comes from one static device array of
 * FLR_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps until the
 * process exits.  The first call on a device looks up that array's device
 * address (with that device current) and caches it; make that first call
 * before any stream capture.  Every call shares the array and it keeps the
 * previous call's contents (what must start at zero is cleared on each
 * call); calls whose GPU work overlaps -- on other streams or from other
 * threads -- race on it and must be serialised by the caller.
 *
 *   Xt        X stored column-major, device memory: column j (n values) starts
 *             at element j*ldn.  ldn >= n, ldn * element size a multiple of 16
 *             bytes, Xt 16-byte aligned; elements in rows n..ldn-1 must be
 *             finite (zero is typical).  dtype as in flr_create.
 *   y         n doubles, device memory.
 *   E         FLR_E_CHAIN or FLR_E_LATTICE (FLR_E_EDGES: FLR_ENOTIMPL).
 *   lambda1, lambda2, eps, tol, opts: as in flr_solve (beta starts at
 *             X_j^T y / X_j^T X_j).
 *   beta_out  p doubles, device memory.
 *   stream    cudaStream_t all work is issued on; the call returns when done.
 *   stats     optional, host memory (ms is host wall time).
 * Scratch needed, in bytes, with every term rounded up to a multiple of 256:
 *     256 + 32768 + 256 + 7 * (8*p) + 2 * (8*ldn)
 *   + 8 * (8*p)        with FLR_PC_TWOLEVEL (what FLR_PC_AUTO selects)
 *   + 2 * (8*p*L)      with the chunk-tridiagonal solve (FLR_PC_TRIDIAG,
 *                      FLR_PC_PAPER, and FLR_PC_TWOLEVEL on a chain),
 * where L = ceil(log2(ceil(p / grid))) and grid is the block count of the
 * launch (at most the number of SMs).  So the default on a chain takes
 * about (15 + 2L) * 8 * p bytes.  A problem that needs more than
 * FLR_NOALLOC_SCRATCH_BYTES returns FLR_ESCRATCH before any GPU work.
 * Other errors as flr_solve. */
flr_status flr_solve_noalloc(const void* Xt, int32_t dtype, int64_t n, int64_t p, int64_t ldn,
                             const double* y, const flr_graph* E, double lambda1, double lambda2,
                             double eps, double tol, const flr_opts* opts, double* beta_out,
                             void* stream, flr_stats* stats);


/* ---------------------------------------------------------------------------
 * Serving: a request loop that keeps several FLR fits on the GPU at once.
 * (Deployment layer; the paper solves one problem at a time.)
 *
 * Requests (X, y, E, lambdas) are queued by flr_server_submit.  `slots`
 * worker threads each own a CUDA stream; a free worker admits the oldest
 * queued request whose device-memory footprint fits in what is left of
 * `hbm_budget`, creates its handle on the slot's stream (or reuses the slot's
 * resident handle for the same data_id), solves it with at most
 * `grid_per_slot` thread blocks, copies beta to the server and frees (or
 * keeps) the handle.  Requests that arrive while others run are admitted as
 * slots and memory free up, and their kernels run concurrently on the device.
 * The server's solves hold at most slots * grid_per_slot (<= number of SMs)
 * thread blocks at once, one per SM, which keeps every cooperative solve
 * co-resident: a problem too wide for grid_per_slot blocks (each block's
 * slab of coefficients must fit its shared-memory vectors) takes as many
 * blocks as it needs from that budget.  Solves take blocks in arrival order;
 * while the oldest waiting one cannot run, later ones that fit in the free
 * blocks may overtake it during its first 2 seconds of waiting.  A request's
 * X, y and edges are borrowed: they must stay valid until flr_server_wait has
 * returned for it.
 * ------------------------------------------------------------------------- */
typedef struct flr_server flr_server;
typedef flr_server* flr_server_t;

typedef struct flr_server_opts {
    int32_t slots;          /* concurrent solves (default 4) */
    int32_t grid_per_slot;  /* thread blocks per solve (default SMs / slots) */
    int64_t hbm_budget;     /* bytes of device memory the server may hold (default 3/4 of free) */
    int32_t reserved[8];
} flr_server_opts;

typedef struct flr_request {
    const void* X;          /* n x p row-major, dtype, row stride ldx (as flr_create) */
    int32_t dtype;
    int32_t mem;            /* FLR_MEM_HOST or FLR_MEM_DEVICE for X, y and E->edges */
    int64_t n, p, ldx;
    const double* y;
    flr_graph E;
    double lambda1, lambda2, eps, tol;
    flr_opts opts;          /* opts.grid is capped at grid_per_slot */
    int32_t use_opts;       /* 0: defaults */
    int32_t reserved;
    uint64_t data_id;       /* 0, or an id the caller gives every request with the same X, y
                               and E (a lambda path, repeated fits): a slot keeps the handle
                               of its last such request resident (X already copied to its
                               column-major layout, X^T y and diag(X^T X) computed) and
                               reuses it for the next request with the same id, which then
                               reads none of its own X, y, E.  A resident handle's memory
                               stays counted against hbm_budget until the slot drops it:
                               for a request with another id, or when queued work does not
                               fit otherwise. */
} flr_request;

typedef struct flr_result {
    int32_t status;         /* flr_status of the solve */
    int32_t slot;           /* worker that ran it */
    flr_stats stats;
    double t_submit, t_start, t_end;   /* seconds since the server was created */
    int64_t footprint;      /* device bytes reserved for the request */
    uint64_t dev_t0_ns, dev_t1_ns;     /* the GPU's global timer (ns) when the solve kernel
                                          started and finished; comparable between requests */
    int32_t reused;         /* 1 when the request ran on a slot's resident handle (data_id) */
    int32_t reserved2;
} flr_result;

/* Start a server on the current device (opts may be NULL). */
flr_status flr_server_create(const flr_server_opts* opts, flr_server_t* out);
/* Queue a request; FLR_EINVAL for malformed requests, FLR_ENOMEM when its
 * footprint exceeds the whole budget (refused, never admitted). */
flr_status flr_server_submit(flr_server_t s, const flr_request* req, uint64_t* id);
/* 1 in *done once the request has finished. */
flr_status flr_server_poll(flr_server_t s, uint64_t id, int32_t* done);
/* Block until the request has finished; copies beta (p doubles, host memory;
 * NULL to skip) and the result record, then forgets the request.  Returns the
 * request's status; FLR_EINVAL for an unknown id. */
flr_status flr_server_wait(flr_server_t s, uint64_t id, double* beta_out, flr_result* res);
/* Finish every queued request, stop the workers, release the server. */
flr_status flr_server_destroy(flr_server_t s);
/* Device bytes flr_create + flr_solve need for a problem (admission estimate). */
int64_t flr_footprint(int64_t n, int64_t p, int64_t m, int32_t dtype, int32_t mem);

#ifdef __cplusplus
}
#endif
#endif /* FLR_H */
