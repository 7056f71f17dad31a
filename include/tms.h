/*
 * tms.h -- C ABI of the GB300 (sm_103a) mesh-vs-mesh intersection search.
 *
 * The library finds every intersecting pair of triangles between two
 * triangulated 2D surfaces in R^4 -- a torus's unstable-manifold mesh W^u and
 * another torus's stable-manifold mesh W^s -- following arXiv 2109.14814,
 * Sec. 6 ("Rapid GPU-Assisted Search for Manifold Intersections"): a broad
 * phase (uniform grid over a trimmed world box, per-face axis-aligned bounding
 * boxes, optional Moller quick test) followed by a narrow phase that solves the
 * 4x4 linear system of Eq. (precise) for the barycentric pair (a, b, c, d).
 *
 * Conventions shared by every entry point
 *   - Every pointer marked "device" must point to memory of the CUDA device that
 *     is current on the calling thread.  The caller owns all input and output
 *     buffers; the library owns only the scratch it allocates internally, which
 *     is cached per stream and released by tms_release_workspace() or
 *     tms_destroy_mesh().
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All work
 *     is ordered on that stream.
 *   - Entry points return a tms_status; no C++ exception crosses the ABI.
 *     On an error other than TMS_ERR_CAPACITY the outputs are unspecified.
 *   - The library never falls back to a CPU implementation.
 *
 * Mesh layout (Sec. 6.1 and Sec. 6.3): four coordinate arrays x, y, px, py,
 * each holding N*M float64 values column-major with theta fastest:
 * coordinate of vertex W(theta_i, s_k) at [k*N + i], theta_i = 2*pi*i/N.
 * Quads Q_ik join (i, k), (i+1, k), (i, k+1), (i+1, k+1) with i+1 taken modulo
 * N on a periodic mesh (Sec. 6.1: the theta index wraps around).
 * Each quad is split into two triangles along the (i+1, k)-(i, k+1) diagonal
 * with the vertex orderings of Sec. 6.2.4:
 *   T1: x1 = W(i+1, k), x2 = W(i, k),     x3 = W(i, k+1)
 *   T2: x1 = W(i, k+1), x2 = W(i+1, k+1), x3 = W(i+1, k)
 * Within a mesh view of vertex columns [k0, k1), quad (i, k) (k relative to
 * k0) has id q = k*N + i and its triangles have ids t = 2*q (T1), 2*q + 1 (T2).
 * A quad hit is derivable from a triangle hit as q = t >> 1 (Sec. 6.2: a quad
 * pair intersects iff one of its four triangle pairs does).
 */
#ifndef TMS_H
#define TMS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int tms_status;
enum {
    TMS_OK = 0,
    TMS_ERR_ARG = 1,       /* bad size, range, pointer, or non-finite vertex */
    TMS_ERR_CAPACITY = 2,  /* output buffer too small; required count reported */
    TMS_ERR_TIMEOUT = 3,   /* a bounded device-side wait ran out */
    TMS_ERR_CUDA = 4,      /* a CUDA runtime call failed */
    TMS_ERR_STATE = 5      /* call sequence error (e.g. destroyed handle) */
};

/* Opaque mesh view.  Borrows the caller's device coordinate arrays (it never
 * copies or frees them); owns a device copy of s_k and small metadata. */
typedef struct tms_mesh_s *tms_mesh;

/*
 * tms_build_mesh -- describe one manifold half-layer mesh.  A half-layer is a
 * contiguous range of s columns of the full vertex arrays (Sec. 6.2), so the
 * view is zero-copy.
 *   dX, dY, dPx, dPy : device, N*M float64 each, layout above.  Borrowed: they
 *                      must stay valid and unchanged while the handle is used.
 *   N                : theta samples, N >= 3 (periodic) or N >= 2 (open strip).
 *   M                : s samples in the full arrays.
 *   k0, k1           : vertex columns [k0, k1) form the view; 0 <= k0,
 *                      k1 <= M, k1 - k0 >= 2.
 *   s                : host or device, M strictly increasing float64 values s_k
 *                      (copied; used for the (theta, s) estimates).
 *   periodic_theta   : 1 = the paper's mesh (quads i = 0..N-1, i+1 mod N);
 *                      0 = open strip (quads i = 0..N-2).
 *   stream           : stream used for the s_k copy.
 *   out              : receives the handle.
 * Errors: TMS_ERR_ARG for any size/range violation, NULL pointer, or s not
 * strictly increasing; TMS_ERR_CUDA on a failed allocation/copy.
 * Non-finite vertex coordinates are reported by the search (TMS_ERR_ARG).
 */
tms_status tms_build_mesh(const double *dX, const double *dY, const double *dPx,
                          const double *dPy, int N, int M, int k0, int k1,
                          const double *s, int periodic_theta, void *stream,
                          tms_mesh *out);

/* Releases the handle and any cached search plan that refers to it.
 * Synchronises the device first. */
tms_status tms_destroy_mesh(tms_mesh mesh);

/* Search parameters.  Fill with tms_params_default() and override fields. */
typedef struct {
    int precision;        /* broad-phase arithmetic: 0 = FP64 boxes and cell keys
                             (plain); 1 = FP32 boxes rounded outward and FP32 cell
                             keys (mixed, default).  The narrow phase is FP64. */
    int face_level;       /* 0 = one box per triangle; 1 = one box per quad, as
                             the paper's kernel (4 triangle pairs per candidate;
                             default). */
    int moller;           /* 1 = apply the Moller quick test of Sec. 6.2.3 (FP64,
                             with a rounding guard) to candidates; default 0.
                             Like the boxes, it is not widened by tau. */
    int cell_filter;      /* 1 = register only faces in grid cells occupied by
                             both meshes before grouping (default); 0 = emit
                             every face-cell incidence (the paper's per-box lists). */
    int narrow_filter;    /* 1 = reject candidates the FP32 tests prove are no
                             FP64 hit: separating axes against the FP64 solve's
                             backward error, and a verified FP32 solve whose
                             error bound certifies margin < -2 tau (default);
                             undecided candidates get the FP64 solve. */
    float cell_mult;      /* grid cell edge = cell_mult x widest face extent per
                             coordinate (Sec. 6.2.1 requires > 1 x); default 1.0625 */
    double tau;           /* margin tolerance of the hit test, default 1e-12; it
                             widens the hit test (weights >= -tau), not the broad
                             phase, whose boxes are the faces' own: meant for
                             tolerances of the order of the rounding */
    long long entry_capacity;  /* initial scratch sizes (0 = automatic); grown on */
    long long cand_capacity;   /* overflow and retried inside the call          */
    long long hit_capacity;    /* raw hits before merging (0 = automatic)       */
    int use_graph;        /* 1 = capture the launch sequence in a CUDA graph on
                             first use and replay it (default 1) */
    unsigned inject;      /* fault injection for tests:
                             bit0 = force entry capacity 1 (exercises retry),
                             bit1 = force a capacity error to be returned,
                             bit2 = report TMS_ERR_TIMEOUT from the host,
                             bit3 = start the cell table at 1024 slots (exercises
                             its growth),
                             bit4 = on the device, the hit sort's look-back reads
                             every earlier tile as not yet published, so each of
                             its bounded waits runs out after spin_limit polls
                             (no fault: the kernel records ST_TIMEOUT, keeps its
                             writes in bounds and returns; TMS_ERR_TIMEOUT),
                             bit5 = start the patch-pair, candidate, survivor and
                             raw-hit buffers at one record (exercises each growth
                             and its retry) */
    int block_faces;      /* bounds-pass tile width in quads (64/128/256; 0 = 128) */
    int tile_rows;        /* bounds-pass tile height in quad rows (4 or 8; 0 = 4) */
    int timing;           /* 1 = record CUDA events between stages (in the graph) so
                             that tms_last_stage_ms() reports per-stage device time */
    int patch;            /* broad-phase level: 0 = the grid holds the faces
                             themselves; 1 = the grid holds patches of 8 x 4 quads
                             (their boxes the union of the quads'), and the quad
                             pairs of every patch pair whose boxes overlap are
                             tested in one warp tile (quad faces only; ignored
                             with face_level 0).  Same candidates either way. */
    int pad0;
    long long spin_limit; /* polls of one device-side wait before it gives up
                             (ST_TIMEOUT, TMS_ERR_TIMEOUT); 0 = 4194304 */
    const char *autotune_cache; /* NULL, or a cache file written by tms_autotune:
                             when it holds an entry for these meshes' size class
                             (see tms_autotune), that entry's face level, cell
                             size, patch level and bounds-pass tile replace the
                             fields given here; read on the first search of a
                             plan only */
} tms_params;

void tms_params_default(tms_params *p);

/* One hit: an intersecting triangle pair (Sec. 6.2.4) and its estimates. */
typedef struct {
    uint32_t triA, triB;   /* triangle ids in mesh A and mesh B */
    uint32_t pair;         /* mesh-pair index (0 for tms_search) */
    uint32_t flags;        /* bit0: near-degenerate band (rho < 1e-12 or
                              |margin| < 1e-12); bit1: the point lies on a shared
                              edge or vertex (this record is the representative) */
    double a, b, c, d;     /* solution of Eq. (precise) */
    double P[4];           /* x-side point x2 + a(x1-x2) + b(x3-x2) */
    double theta_u, s_u;   /* estimates on mesh A, Sec. 6.2.4 (theta in [0, 2pi)) */
    double theta_s, s_s;   /* estimates on mesh B */
    double rho;            /* |det| / product of the column norms */
    double margin;         /* min(a, b, c, d, 1-a-b, 1-c-d) */
} tms_hit;

/*
 * tms_search -- all intersecting triangle pairs of mesh A against mesh B.
 *   params   : may be NULL (defaults).
 *   dHits    : device, room for hitCap records (may be NULL when hitCap is 0).
 *   hitCap   : capacity of dHits in records.
 *   nHits    : host out; the number of hits.  On TMS_ERR_CAPACITY it holds the
 *              required count and dHits holds the first hitCap records.
 * Output order: sorted by (triA, triB); hits on shared edges/vertices merged
 * (one record per feature pair, the smallest (triA, triB)).  Deterministic.
 * Synchronises `stream` before returning (to read the count).
 */
tms_status tms_search(tms_mesh A, tms_mesh B, const tms_params *params,
                      tms_hit *dHits, long long hitCap, long long *nHits,
                      void *stream);

/*
 * tms_search_host -- tms_search for meshes whose coordinates are given in host
 * memory: copies the view rows [k0, k1) of both meshes' four coordinate arrays
 * from host memory into the device arrays the meshes were built on, searches,
 * and copies the merged hits to host memory; returns when they are there.
 *   hostA, hostB : host, four pointers each (x, y, px, py), each a full M x N
 *                  array in the layout of the device arrays (vertex (i, k) at
 *                  k*N + i); pinned memory copies fastest.  The device arrays
 *                  are overwritten with them.
 *   hostHits     : host, room for hitCap records; nHits as in tms_search.
 *   stream       : the copies and the search are ordered on it.
 * The device output lives in a per-device buffer of the library, grown on
 * demand (the first call for a larger hitCap allocates).  Errors as
 * tms_search; TMS_ERR_ARG for a NULL pointer.
 */
tms_status tms_search_host(tms_mesh A, const double *const hostA[4], tms_mesh B,
                           const double *const hostB[4], const tms_params *params,
                           tms_hit *hostHits, long long hitCap, long long *nHits,
                           void *stream);

/*
 * tms_search_batched -- nPairs independent searches (A[p], B[p]) of uneven
 * sizes in one launch sequence: every stage is one persistent launch over all
 * pairs' work, and the sequence is captured once into a CUDA graph and replayed
 * while the handles, params and output pointers are unchanged.
 *   dHits    : device, hitCap records; hits of all pairs, sorted by
 *              (pair, triA, triB).
 *   dOffsets : device, nPairs+1 int64; hits of pair p are
 *              dHits[dOffsets[p] .. dOffsets[p+1]).
 *   nHits    : host out, total count (required count on TMS_ERR_CAPACITY).
 */
tms_status tms_search_batched(const tms_mesh *A, const tms_mesh *B, int nPairs,
                              const tms_params *params, tms_hit *dHits,
                              long long hitCap, long long *dOffsets,
                              long long *nHits, void *stream);

/*
 * tms_backward -- reverse-mode derivative of hit outputs with respect to the
 * mesh vertices and a family parameter alpha, by implicit differentiation of
 * A z = r (Eq. (precise)): with zbar = gZ + (dP/dz)^T gP and w = A^{-T} zbar,
 * the vertex gradients are x_i: beta_i (gP - w), y_i: gamma_i w with barycentric
 * weights beta = (a, 1-a-b, b), gamma = (c, 1-c-d, d) on (x1, x2, x3), (y1, y2, y3).
 *   dHits            : device, nHits records from tms_search (triA, triB used).
 *   dGradP, dGradZ   : device, nHits*4 float64 upstream gradients on P and
 *                      (a, b, c, d); either may be NULL (= zeros).
 *   dGradA, dGradB   : device, 4*N*M float64 each (layout of the mesh arrays,
 *                      full M); ACCUMULATED into (atomic adds); may be NULL.
 *   dDvDalphaA/B     : device, 4*N*M float64 d(vertex)/d(alpha), or NULL.
 *   dGradAlpha       : device, nHits float64, written (not accumulated):
 *                      per-hit sum over its six vertices of grad . dv/dalpha;
 *                      may be NULL.
 * Hits whose system is singular contribute nothing.
 */
tms_status tms_backward(tms_mesh A, tms_mesh B, const tms_hit *dHits, long long nHits,
                        const double *dGradP, const double *dGradZ,
                        double *dGradA, double *dGradB,
                        const double *dDvDalphaA, const double *dDvDalphaB,
                        double *dGradAlpha, void *stream);

/*
 * tms_autotune -- picks, for these meshes, the search parameters the paper
 * leaves to the implementation (Sec. 6.2.1 grid cell size; Sec. 6.3 launch
 * shape): face level (quads or triangles), cell_mult in {1.0625, 1.5, 2.5},
 * block_faces in {64, 128} and tile_rows in {4, 8}, by timing each of the 24
 * settings (one warm-up and three timed runs, median) with tms_search (nPairs == 1) or
 * tms_search_batched (nPairs > 1) on `stream`.  The other fields (precision,
 * filters, tau, capacities, use_graph) come from `base` (NULL = defaults) and
 * are kept.  Results are unchanged by the choice: every setting finds the same
 * hits.
 *   A, B       : nPairs mesh handles each (host arrays).
 *   best       : host out, `base` with the four fields set to the fastest.
 *   cache_path : text file, or NULL for no cache.  A line per tuned key
 *                "<device>|pairs=..|sizes=<hash of every N,M>|prec=..|... fl cm bf tr ms";
 *                a matching line is returned without timing anything; a new
 *                result is appended.
 *   best_ms    : host out (may be NULL), median time of the chosen setting.
 * Allocates trial output buffers with cudaMalloc and frees them, releases the
 * trial plans of `stream` between settings, synchronises.  TMS_ERR_ARG on NULL
 * handles or nPairs <= 0; a setting that fails is skipped; TMS_ERR_CUDA when
 * none succeeds.
 */
tms_status tms_autotune(const tms_mesh *A, const tms_mesh *B, int nPairs,
                        const tms_params *base, tms_params *best, const char *cache_path,
                        double *best_ms, void *stream);

/* Per-stage statistics of the last search on `stream` (host copies). */
typedef struct {
    long long entries;      /* face-cell entries (grouped by cell) */
    long long cells;        /* occupied cells holding both meshes */
    long long pair_slots;   /* sum over cells of nA*nB */
    long long candidates;   /* candidate face pairs after box and owner tests */
    long long fp64_solves;  /* triangle pairs sent to the FP64 solve */
    long long raw_hits;     /* hits before merging */
    long long hits;         /* output hits */
    int grid_n[4];          /* cells per coordinate (pair 0) */
    int empty;              /* trimmed world empty (pair 0) */
    int retries;            /* capacity retries taken */
    int kernels;            /* kernel launches in one search (graph replay) */
    int pad;
    long long fp32_solves;  /* triangle pairs through the verified FP32 solve */
    long long sat_tests;    /* triangle pairs through the separating-axis prefilter */
    long long quad_tests;   /* quad candidates through the quad-level prefilter */
    long long patch_pairs;  /* patch level: patch pairs with overlapping boxes */
    long long patch_tests;  /* patch level: quad pairs box-tested inside them */
    long long quad_kept;    /* quad candidates the quad-level test could not clear */
    long long patch_kept;   /* patch level: patch pairs with an overlapping quarter pair */
} tms_stats;

tms_status tms_last_stats(void *stream, tms_stats *out);

/*
 * tms_search_noalloc -- tms_search for callers that must not allocate device
 * memory.  The paper has no counterpart: this is a deployment variant.
 * Callers that cannot call cudaMalloc include real-time or flight software
 * that fixes its device footprint at start-up and forbids allocation later,
 * services whose device memory is entirely held by a pool allocator (a direct
 * cudaMalloc fails or fragments the pool), and embedded hosts that budget
 * every device byte when they start.  Every scratch buffer comes from one
 * file-scope static __device__ array of 72 MiB that every GPU loading this
 * library holds until the process exits; the call makes no cudaMalloc,
 * cudaFree or other allocating call.  Arguments, output order and merging are
 * those of tms_search.  Limits: each mesh view at most 131072 vertices
 * (TMS_ERR_ARG otherwise); at most 262144 face-cell entries, 262144
 * candidates, 65536 FP64 solves and 16384 hits before merging
 * (TMS_ERR_CAPACITY, *nHits = -1, when a stage overflows; nothing is grown).
 * All calls share the array, which keeps the last call's contents; each call
 * clears what must start at zero, and a call that overflows leaves the array
 * fit for the next.  Calls whose GPU work overlaps (two streams, two host
 * threads) race on the array and must be ordered by the caller.  The first
 * call on a device looks up the array's device address with that device
 * current and configures the kernels: make it before any stream capture.
 * Synchronises `stream`.  Every error return sets a message, read with
 * tms_noalloc_last_error().
 */
tms_status tms_search_noalloc(tms_mesh A, tms_mesh B, const tms_params *params,
                              tms_hit *dHits, long long hitCap, long long *nHits,
                              void *stream);
const char *tms_noalloc_last_error(void);

/* Bytes of the static array the layout of tms_search_noalloc uses (*needed)
 * and holds (*reserved); host only, no device call.  A build whose layout
 * does not fit refuses every call with TMS_ERR_STATE. */
tms_status tms_noalloc_footprint(unsigned long long *needed, unsigned long long *reserved);

/*
 * Method of layers (Sec. 5, Eq. layerintersection; Sec. 6.2).  With the
 * fundamental domains (-D_u, D_u), (-D_s, D_s) and multipliers lam_u > 1,
 * 0 < lam_s < 1, the half-layers are
 *   U_n^+- = W^u(T x +-[D_u lam_u^(n-1), D_u lam_u^n]),
 *   S_m^+- = W^s(T x +-[D_s / lam_s^(m-1), D_s / lam_s^m]),
 * and every heteroclinic orbit has a point in some U_n cap S_n or
 * U_n cap S_(n-1), n >= 1.  On globalized meshes whose stored s values include
 * the boundaries, a half-layer is a contiguous range of vertex columns, so
 * each of the 8 pairs of a layer is one search between two mesh views.
 */
typedef struct {
    int n, m;             /* U_n and S_m, m = n or n - 1 */
    int sign_u, sign_s;   /* +1 or -1: positive or negative half-layer */
    int a_k0, a_k1;       /* vertex columns [a_k0, a_k1) of U_n^sign_u in A's arrays */
    int b_k0, b_k1;       /* vertex columns [b_k0, b_k1) of S_m^sign_s in B's arrays */
} tms_layer_pair;

/*
 * tms_layer_pairs -- the 8 n_max half-layer pairs for layers 1..n_max, in the
 * order n ascending, then sign_u (+1 first), then m = n before m = n - 1, then
 * sign_s (+1 first).  Host only, no device call.
 *   sA, sB   : host, MA and MB strictly increasing s values of the full meshes.
 *   rel_tol  : a boundary value b matches the stored s_k with |s_k - b| <= rel_tol |b|.
 *   out, cap : host, room for cap pairs; *count receives 8 n_max.
 * TMS_ERR_ARG when a boundary is not a stored value (message names the layer)
 * or an argument is out of range; TMS_ERR_CAPACITY when cap < 8 n_max (the
 * first cap pairs are written).
 */
tms_status tms_layer_pairs(const double *sA, int MA, double Du, double lam_u, const double *sB,
                           int MB, double Ds, double lam_s, int n_max, double rel_tol,
                           tms_layer_pair *out, int cap, int *count);

/* A layer sweep: one mesh view per distinct half-layer of the full meshes A
 * and B (borrowing their arrays, like tms_build_mesh) and the per-pair id
 * shifts.  The pairs' column ranges are indices into the arrays A and B were
 * built on and must lie inside their views.  Creating it synchronises. */
typedef struct tms_layer_plan_s *tms_layer_plan;
tms_status tms_layer_plan_create(tms_mesh A, tms_mesh B, const tms_layer_pair *pairs,
                                 int nPairs, void *stream, tms_layer_plan *out);
tms_status tms_layer_plan_destroy(tms_layer_plan plan);

/*
 * tms_layer_search -- every intersecting triangle pair of every half-layer
 * pair of the plan, as one tms_search_batched over the views (one graph
 * replay), with triangle ids shifted to the views of A and B the plan was
 * made from (so they are unique across pairs).  Output as tms_search_batched:
 * sorted by (pair, triA, triB), pair = index into the plan's pairs, dOffsets
 * (device, nPairs + 1) required.  The id shift runs on `stream` after the
 * search's own synchronisation.  TMS_ERR_CAPACITY as tms_search_batched (the
 * first hitCap records are shifted too).
 */
tms_status tms_layer_search(tms_layer_plan plan, const tms_params *params, tms_hit *dHits,
                            long long hitCap, long long *dOffsets, long long *nHits, void *stream);

/*
 * Refinement of approximate intersections (Sec. 7, Eqs. tosolve and
 * dampedNewtonEquation).  Each seed x0 = (theta_u, s_u, theta_s, s_s) -- for
 * example a hit's parameter estimates (Sec. 6.2.4) -- is corrected by the
 * damped Newton iteration x_{k+1} = x_k - alpha Df(x_k)^{-1} f(x_k) on
 *     f(x) = W_A(theta_u, s_u) - W_B(theta_s, s_s),
 *     Df   = [df/dtheta_u, df/ds_u, df/dtheta_s, df/ds_s]   (4x4, FP64),
 * evaluated on the true surfaces rather than their meshes.  The paper obtains
 * W and its partials from Fourier-Taylor series and the flow
 * (Eqs. wuequation-dwsdsequation); this library evaluates the closed-form
 * sheet pair below, which its synthetic meshes sample, with exact partials.
 *
 * The sheet pair (all lengths 4 = the coordinates x, y, px, py):
 *   S(theta, s; a)  = g(s) T(theta; a) + F(s)
 *   T(theta; a)     = sum_{k=1..K} ((ca_k + a dca_k) cos k theta
 *                                   + (cb_k + a dcb_k) sin k theta) / k
 *   g(s)            = 1 + s (stretch 0) or lam^s (stretch 1)
 *   F(s)            = sum_f fold_amp_f (s - r_f1)(s - r_f2)(s - r_f3) fold_dir_f
 *   W_A(theta, s)   = S(theta, s; alpha_u)
 *   W_B(theta, s)   = S(theta + c0, 1 - s; alpha_s)
 *                     + h_amp (sin(P (theta - theta0)) n1 + sin(Q pi (s - s0)) n2)
 *   n_r(theta, s)   = v_r - t1 y1 - t2 y2,  (y1, y2) = (J^T J + eps I)^{-1} J^T v_r,
 *                     J = [t1 t2] = the theta- and s-partials of
 *                     S(theta', s'; alpha_ref) at theta' = theta + c0, s' = 1 - s,
 *                     eps = reg (|t1|^2 + |t2|^2) / 2.
 */
#define TMS_SURF_MAX_HARMONICS 8
#define TMS_SURF_MAX_FOLDS 4

typedef struct {
    int n_harmonics;            /* K, 1..TMS_SURF_MAX_HARMONICS */
    int n_folds;                /* 0..TMS_SURF_MAX_FOLDS */
    int stretch;                /* 0: g = 1 + s; 1: g = lam^s */
    int pad;
    double ca[TMS_SURF_MAX_HARMONICS][4];    /* row k-1 holds harmonic k */
    double cb[TMS_SURF_MAX_HARMONICS][4];
    double dca[TMS_SURF_MAX_HARMONICS][4];   /* derivatives in the family parameter */
    double dcb[TMS_SURF_MAX_HARMONICS][4];
    double alpha_u;             /* family parameter of W_A (the paper's omega_u) */
    double alpha_s;             /* family parameter of B's sheet (omega_s) */
    double alpha_ref;           /* family parameter of the normal frame */
    double lam;                 /* stretch base (stretch 1), > 0 */
    double fold_amp[TMS_SURF_MAX_FOLDS];
    double fold_root[TMS_SURF_MAX_FOLDS][3];
    double fold_dir[TMS_SURF_MAX_FOLDS][4];
    double c0;                  /* theta offset of B's underlying sheet */
    double h_amp, P, Q;         /* crossing term amplitude and frequencies */
    double theta0, s0;          /* crossing lattice origin */
    double v1[4], v2[4];        /* generating directions of the normal frame */
    double reg;                 /* frame regulariser, >= 0 */
} tms_surface_pair;

typedef struct {
    double alpha0;        /* damping while ||f||_2 > switch_below, in (0, 1] */
    double alpha1;        /* damping once ||f||_2 <= switch_below, in (0, 1] */
    double switch_below;  /* >= 0 (0: alpha0 throughout) */
    double tol;           /* converged when ||f(x_k)||_2 <= tol, >= 0 */
    double s_lo, s_hi;    /* a seed whose s_u or s_s leaves [s_lo, s_hi] stops */
    double rho_min;       /* singular when |det Df| / prod_j ||Df e_j|| < rho_min */
    int max_iter;         /* at most this many updates, 0..1000000 */
    int pad;
} tms_refine_params;

/* alpha0 = alpha1 = 0.5, switch_below = 0, tol = 1e-10, s in [-0.5, 1.5],
 * rho_min = 1e-14, max_iter = 200. */
void tms_refine_params_default(tms_refine_params *p);

enum {
    TMS_REFINE_CONVERGED = 0,   /* ||f|| <= tol at the returned x */
    TMS_REFINE_MAX_ITER = 1,    /* max_iter updates made without converging */
    TMS_REFINE_SINGULAR = 2,    /* normalised |det Df| below rho_min */
    TMS_REFINE_ESCAPED = 3,     /* s_u or s_s left [s_lo, s_hi] */
    TMS_REFINE_NON_FINITE = 4   /* a non-finite iterate, f or Df */
};

/*
 * tms_refine -- damped Newton from n seeds, one independent iteration each.
 *   surf, params : host; params may be NULL (defaults).
 *   dX0          : device, seed i at dX0[i*ldx0 + 0..3] = (theta_u, s_u,
 *                  theta_s, s_s); ldx0 >= 4 doubles (16 reads seeds straight
 *                  out of tms_hit records: dX0 = (const double *)dHits + 10).
 *   dX           : device, n*4 doubles out: the last iterate, theta_u and
 *                  theta_s reduced to [0, 2 pi).  May equal dX0 when ldx0 == 4.
 *   dFnorm       : device, n doubles: ||f||_2 at the last evaluation (NaN when
 *                  the seed stopped before one: escaped or non-finite).
 *   dRho         : device, n doubles: det Df / prod_j ||Df e_j|| at the last
 *                  evaluation (signed; NaN as for dFnorm).
 *   dIters       : device, n int32: updates made.
 *   dStatus      : device, n int32: TMS_REFINE_*.
 *   dFnorm, dRho, dIters, dStatus may be NULL.
 * Checks in order at every iterate: non-finite or escaped x stops; then f and
 * Df are evaluated; non-finite f or Df stops; ||f|| <= tol converges;
 * max_iter updates made stops; a singular Df stops; else x is updated.
 * Asynchronous on `stream`; allocates nothing.  TMS_ERR_ARG on a bad argument
 * (message in tms_last_error()), TMS_ERR_CUDA on a launch failure.
 */
tms_status tms_refine(const tms_surface_pair *surf, const tms_refine_params *params,
                      const double *dX0, long long ldx0, long long n, double *dX,
                      double *dFnorm, double *dRho, int32_t *dIters, int32_t *dStatus,
                      void *stream);

/*
 * Continuation of connections through the torus families (Sec. 8, Eq.
 * predictor): the family parameter alpha_u of W_A (param 0) or alpha_s of B's
 * sheet (param 1) -- the paper's rotation numbers omega_u, omega_s -- walks
 * alpha_0 (the pair's own value), alpha_1, ..., alpha_nSteps while the other is
 * held.  Per branch (one per seed) and step j:
 *   predictor  j = 0: the seed; j = 1: x_0;
 *              j >= 2: x_{j-1} + (alpha_j - alpha_{j-1}) / (alpha_{j-1} - alpha_{j-2})
 *                                (x_{j-1} - x_{j-2}), angle differences in [-pi, pi]
 *              (consecutive parameter values must differ);
 *   corrector  tms_refine's damped Newton at alpha_j (params.corrector);
 *   monitor    a converged step whose point lies farther than max_jump from its
 *              prediction in some coordinate (angles on the circle) is
 *              TMS_CONT_JUMPED; else one whose normalised det Df is below
 *              rho_turn in magnitude or of the other sign than at step j-1 is
 *              TMS_CONT_TURNING (a fold of the branch).
 * A branch stops at its first step that is not TMS_REFINE_CONVERGED (the
 * corrector's status, TURNING or JUMPED; that step's x is kept); its later
 * steps are TMS_CONT_STOPPED with NaN outputs.
 */
enum {
    TMS_CONT_TURNING = 5,
    TMS_CONT_JUMPED = 6,
    TMS_CONT_STOPPED = 7
};

typedef struct {
    tms_refine_params corrector;  /* damped Newton of every step */
    double rho_turn;              /* >= 0 */
    double max_jump;              /* > 0 */
    int param;                    /* 0: continue in alpha_u; 1: in alpha_s */
    int pad;
} tms_continue_params;

/* corrector = tms_refine_params_default(), rho_turn = 1e-8, max_jump = 0.25,
 * param = 0. */
void tms_continue_params_default(tms_continue_params *p);

/*
 * tms_continue -- nBranches independent continuations.
 *   surf, params : host; params may be NULL (defaults).
 *   dAlphas      : device, nSteps parameter values alpha_1..alpha_nSteps
 *                  (may be NULL when nSteps is 0).
 *   dX0          : device, seed b at dX0[b*ldx0 + 0..3], ldx0 >= 4.
 *   dX           : device, nBranches*(nSteps+1)*4 doubles: step j of branch b
 *                  at [(b*(nSteps+1) + j)*4], angles in [0, 2 pi).
 *   dStatus      : device, nBranches*(nSteps+1) int32 (TMS_REFINE_*, TMS_CONT_*).
 *   dIters, dRho, dFnorm : device, same count, or NULL: corrector updates, det Df /
 *                  prod of column norms and ||f||_2 at the step's last evaluation.
 * Asynchronous on `stream`; allocates nothing.  TMS_ERR_ARG on a bad argument,
 * TMS_ERR_CUDA on a launch failure.
 */
tms_status tms_continue(const tms_surface_pair *surf, const tms_continue_params *params,
                        const double *dAlphas, int nSteps, const double *dX0, long long ldx0,
                        long long nBranches, double *dX, int32_t *dStatus, int32_t *dIters,
                        double *dRho, double *dFnorm, void *stream);

/*
 * Operations on theta grids (functions of theta stored at theta_i = 2 pi i / N,
 * Sec. 4 and Sec. 6.1).
 *
 * tms_theta_translate -- Eq. (translate): every column of a coordinate array
 * replaced by the samples of its trigonometric interpolant at theta_i + rho
 * (FFT, multiply the k-th coefficient by e^{j k rho}, inverse FFT); with
 * derivative = 1, by those of its theta-derivative at theta_i + rho (the
 * coefficient times j k e^{j k rho}, Eq. translate2).  k runs over the signed
 * frequencies -N/2 < k < N/2; the Nyquist coefficient is multiplied by
 * cos(N rho / 2) (0 for the derivative), so real data stay real.  Globalizing
 * a manifold (Sec. 6.1) translates each s column by rho = -n omega.
 *   dIn, dOut : device, nCoord blocks of nCols columns of N doubles (theta
 *               fastest; block c at c * ldc, column k at c * ldc + k * N) --
 *               the mesh layout.  dOut may equal dIn.
 *   N         : power of two, 8..8192.
 *   dRho      : device, nCols shifts (one per column, shared by its
 *               coordinates), or NULL to use rho0 for every column.
 * FP64 throughout.  Asynchronous; allocates nothing.  TMS_ERR_ARG on a bad
 * size or pointer.
 */
tms_status tms_theta_translate(const double *dIn, double *dOut, int N, int nCols, int nCoord,
                               long long ldc, const double *dRho, double rho0, int derivative,
                               void *stream);

/*
 * tms_phase_align -- Eq. (rhoEquationDiscrete) for nAlign independent pairs of
 * circles: cost(m) = sum_i || Wr(theta_i + 2 pi m / N) - Wprev(theta_i) ||
 * (Euclidean norm over the nCoord coordinates; Wr(theta_i + 2 pi m / N) is the
 * sample (i + m) mod N) for m = 0..N-1, and its minimiser (ties to the
 * smallest m).  The paper aligns each torus of a family with the previous,
 * already aligned one; since a grid shift only reindexes, aligning every
 * consecutive raw pair at once and summing the shifts gives the same result.
 *   dWr, dWprev : device, nAlign x nCoord x N doubles (alignment a at
 *                 a * nCoord * N, coordinate c at + c * N).  1 <= nCoord <= 8.
 *   dCost       : device, nAlign x N doubles out.
 *   dShift      : device, nAlign int32 out: the minimising m.
 * FP64; each cost is summed in order of i.  Asynchronous; allocates nothing.
 */
tms_status tms_phase_align(const double *dWr, const double *dWprev, int N, int nCoord,
                           int nAlign, double *dCost, int32_t *dShift, void *stream);

/* Per-stage device time (ms) of the last search on `stream` made with
 * params.timing = 1, in this order:
 *   0 counters/bounds init   1 face pass: world bounds   2 grid parameters
 *   3 bitmap clear           4 face pass: mark A         5 face pass: probe B
 *   6 face pass: probe A (or emit all)  7 cell table: counts and ranks
 *   8 cells and scatter of the face ids
 *   9 candidate emission (patch level: patch pairs)
 *   10 patch level: quad pairs of the patch pairs (0 otherwise)
 *   11 narrow phase          12 sort hits
 *   13 merge + output        14 counter read-back
 * The face passes, cell table and emission work on patches at the patch
 * level.  Writes min(cap, 15) values; *n receives 15. */
tms_status tms_last_stage_ms(void *stream, float *ms, int cap, int *n);

/* Frees the scratch and cached plans created for `stream`; NULL frees those of
 * every stream.  Synchronises the plans' work first. */
tms_status tms_release_workspace(void *stream);

/* Read-back of the patch frames of the last search on `stream` (patch level,
 * mixed precision, narrow_filter 1), so that tests can check their bounds
 * against the FP64 vertices.  side: 0 = mesh A, 1 = mesh B of pair 0.
 * host_out: host, room for cap floats; receives, per patch in slot order
 * (patch row * npi + patch column), 28 floats: c[4], e_0..e_3 (4 each),
 * h_0..h_3, rho, L, n_2, n_3 -- an FP32 point c, four FP32 axes and bounds
 * that hold for every FP64 vertex V of the patch:
 *   |e_k . (V - c)| <= h_k,  max_i |r_i| <= rho with
 *   r = (V - c) - sum_k (e_k . (V - c)) e_k,  max_i |V_i| <= L,
 *   n_2 >= |e_2|_1,  n_3 >= |e_3|_1
 * (h and rho are +inf on a patch without a usable frame).  The patch-pair
 * test drops a pair when along e_2 or e_3 of either patch, or along a
 * direction orthogonal to e_0, e_1 of one patch and e_0 or e_1 of the other,
 * the two patches' intervals are further apart than the FP64 solve's backward
 * error and the hit tolerance allow (no triangle pair in them can be an FP64
 * hit).
 * *n_patches, *npi (host): patches and patches per quad row.  Synchronises
 * the stream.  TMS_ERR_STATE when no such search was made on `stream`;
 * TMS_ERR_CAPACITY (with the counts set) when cap < 28 * patches. */
tms_status tms_last_patch_frames(void *stream, int side, float *host_out, long long cap,
                                 long long *n_patches, int *npi);

/* Measures this GPU's FP64 fused-multiply-add throughput (TFLOP/s) with a
 * short dependent-chain kernel on `stream`; the denominator of the narrow
 * phase's FP64 utilisation.  Allocates a small buffer; synchronises. */
tms_status tms_probe_fp64(double *tflops, void *stream);

/* Message describing the last error returned on the calling thread. */
const char *tms_last_error(void);

/* Static string for a status code. */
const char *tms_status_str(tms_status s);

/* Library version string. */
const char *tms_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TMS_H */
