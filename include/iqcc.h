/*
 * iqcc.h - C ABI of libiqcc.so, the GB300 (sm_103a) hot path of iterative
 * qubit coupled cluster (iQCC, arXiv 2603.08883).
 *
 * One opaque context owns one qubit Hamiltonian H = sum_k C_k P_k (Eq. 2 /
 * Eq. 9, real C_k) resident in GPU memory, and every operation below runs as
 * CUDA kernels on the context's stream.  No PyTorch type appears here.
 *
 * Pauli keys.  A string on n qubits is stored as two bit vectors x and z of
 * W = ceil(n/64) little-endian 64-bit words (qubit j = bit j%64 of word j/64);
 * the letter of qubit j is (x,z) = (0,0) I, (1,0) X, (1,1) Y, (0,1) Z, and
 * P(x,z) = i^{popcount(x&z)} X^x Z^z is Hermitian.  Arrays of keys are
 * row-major [count][W]; bits at qubits >= n must be zero.  This is the
 * "binary strings of X and Z components" of the paper's GPU section.
 *
 * Sign convention.  iqcc_dress(P, tau) maps H to e^{-i tau P/2} H e^{+i tau P/2}:
 * a string T that anticommutes with P becomes cos(tau) T + sin(tau) (i T P),
 * one that commutes is kept.  This is Eq. 5 with tau = -tau_paper; energies and
 * their minima are the same, gradients flip sign:
 * dE/dtau = -Im<Omega|H P|Omega> (Eq. 7 gives +Im for tau_paper).
 *
 * Canonical key order (export, DIS ties, compression ties): x as an unsigned
 * integer of W words (word W-1 most significant), then z the same way.
 *
 * Memory and calls.  All pointer arguments are HOST memory unless stated.
 * Inputs are copied; the library never keeps or frees caller memory.  Calls
 * are ordered on opts.stream and return after their outputs are written
 * (they synchronise that stream).  A context is used by one host thread at a
 * time.  Device memory comes from opts.alloc/opts.free when given (e.g. a
 * framework's caching allocator), else cudaMalloc/cudaFree; it grows on demand
 * up to opts.capacity rows.
 *
 * Errors.  Every entry point returns an iqcc_status; iqcc_last_error() gives a
 * one-line message.  On IQCC_ERR_ARG nothing was changed.  On
 * IQCC_ERR_CAPACITY the Hamiltonian is exactly as before the generator that
 * would have overflowed (n_applied says how many were applied).  After
 * IQCC_ERR_CUDA, IQCC_ERR_HASH_FULL or IQCC_ERR_TIMEOUT the context is marked
 * broken and later calls return IQCC_ERR_STATE; only iqcc_free() is valid.
 */
#ifndef IQCC_H
#define IQCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct iqcc_ctx iqcc_ctx;

typedef enum {
    IQCC_OK = 0,
    IQCC_ERR_ARG = 1,       /* invalid argument; nothing changed */
    IQCC_ERR_CUDA = 2,      /* CUDA runtime error (context broken) */
    IQCC_ERR_OOM = 3,       /* device allocation failed; H unchanged */
    IQCC_ERR_CAPACITY = 4,  /* a dress would exceed opts.capacity rows; H unchanged */
    IQCC_ERR_HASH_FULL = 5, /* hash probe bound exceeded (context broken) */
    IQCC_ERR_TIMEOUT = 6,   /* a bounded device wait gave up (context broken) */
    IQCC_ERR_STATE = 7      /* context broken by an earlier error */
} iqcc_status;

typedef struct {
    int n_qubits;          /* 1..256 */
    int64_t capacity;      /* maximum number of terms held; 0 -> 1<<30; at most 4294967294 */
    int max_probe;         /* hash buckets probed per lookup (DIS group table, key index of the
                              partitioned dress) before IQCC_ERR_HASH_FULL; 0 -> 64, at most 256 */
    void* stream;          /* cudaStream_t to run on; NULL -> the legacy default stream */
    void* (*alloc)(size_t bytes, void* user); /* device allocator or NULL (cudaMalloc) */
    void (*free)(void* ptr, void* user);      /* matching free or NULL (cudaFree) */
    void* alloc_user;      /* passed to alloc/free */
} iqcc_opts;

/*
 * Create a context holding H = sum_k coef[k] P(x[k], z[k]) (Eq. 2).
 * x, z: host [n_terms][W]; coef: host [n_terms].  Repeated keys are summed in
 * input order and exact zeros are dropped.  Input already in canonical order
 * with distinct keys (an iqcc_export) is checked on the device and kept in
 * that order; other input is grouped by key through a hash partition and a
 * shared-memory join (rows stored in bin order; a device radix sort instead
 * when one string repeats thousands of times).  The row order of a context
 * is not part of its state: iqcc_export returns canonical order regardless.
 * n_terms may be 0.
 * On success *out owns the context (free with iqcc_free); on failure *out is
 * NULL and iqcc_last_error(NULL) describes the error.
 */
iqcc_status iqcc_load_hamiltonian(iqcc_ctx** out, const iqcc_opts* opts, int64_t n_terms,
                                  const uint64_t* x, const uint64_t* z, const double* coef);

/*
 * Dress H in place with n_gen generators, in order k = 0..n_gen-1 (Eq. 5,
 * Eq. 6; App. A procedure step 4), each the Hermitian string P(gx[k], gz[k])
 * with amplitude tau[k] in the convention above.  gx, gz: host [n_gen][W];
 * tau: host [n_gen].  A string T anticommuting with P_k and its partner
 * Q = T xor P_k (i T P_k = s Q, s = +-1) are rotated as a pair when both are
 * present; when Q is absent, T is scaled by cos and Q is appended with
 * s sin(tau) C_T.  Commuting strings are untouched.  Nothing is pruned: exact
 * zeros stay until iqcc_prune.  *n_applied (may be NULL) receives the number
 * of generators applied.
 * The merge (App. D Eq. 18, "insert if unique, else add") is a join: the
 * anticommuting rows are partitioned by a hash of their pair key (of T and
 * T xor P, the one whose bit at P's lowest set bit is clear) and each
 * partition is matched in shared memory; the commuting rows stay in order, the
 * dressed and appended rows follow them.  Device scratch: 16 Wd + 8 bytes per
 * anticommuting row, plus small per-bin arrays.
 * Errors: IQCC_ERR_ARG (bits above n_qubits, non-finite tau),
 * IQCC_ERR_CAPACITY (H as after the previous generator), IQCC_ERR_OOM,
 * IQCC_ERR_CUDA, IQCC_ERR_TIMEOUT (a device wait gave up),
 * IQCC_ERR_HASH_FULL (more than 4096 rows fell into one partition group: far
 * beyond any fluctuation of the hash).
 */
iqcc_status iqcc_dress(iqcc_ctx* ctx, int n_gen, const uint64_t* gx, const uint64_t* gz,
                       const double* tau, int* n_applied);

/*
 * The dress of iqcc_dress by a global sort instead of the partitioned join
 * (the alternative merge of App. D: expansion, sort, segmented reduction).
 * Generators are taken in
 * groups of `fuse` (1..8, the last group may be shorter); each group expands
 * every term along every path through its generators (at generator j a path
 * keeps the current string, with factor cos(tau_j) when it anticommutes with
 * P_j, or, only then, moves to its partner with factor s sin(tau_j)), sorts
 * the expanded terms in canonical key order, sums runs of equal keys in FP64
 * (exact zeros kept) and compacts them.  The result equals iqcc_dress up to
 * rounding (summation order); with fuse > 1 the intermediate merges are
 * skipped.  Terms end in canonical order.
 * gx, gz: host [n_gen][W]; tau: host [n_gen].  Errors: IQCC_ERR_ARG (bad
 * fuse, bits above n_qubits, non-finite tau), IQCC_ERR_CAPACITY when a
 * group's expansion exceeds the capacity (H as after the previous group),
 * IQCC_ERR_OOM, IQCC_ERR_CUDA.  *n_applied (may be NULL): generators applied.
 */
iqcc_status iqcc_dress_sorted(iqcc_ctx* ctx, int n_gen, const uint64_t* gx, const uint64_t* gz,
                              const double* tau, int fuse, int* n_applied);

/*
 * Compress H (App. A procedure step 5; the "Maximum Terms" limit of the
 * paper's Tables 2-3): remove every term with |C| < eps (eps <= 0 removes
 * nothing); then, when max_terms > 0 and more terms remain, keep the max_terms
 * largest |C|, ties at the threshold kept in ascending canonical key order.
 * Surviving terms keep their relative order.  *n_removed may be NULL.
 */
iqcc_status iqcc_prune(iqcc_ctx* ctx, double eps, int64_t max_terms, int64_t* n_removed);

/*
 * iqcc_prune over the union of several contexts on one device, the
 * partitions of one Hamiltonian (App. B): |C| < eps is dropped in every part,
 * then, when max_terms > 0 and more terms remain in all, the max_terms
 * largest |C| of the union are kept, ties at the threshold in ascending
 * canonical key order across the parts (the parts hold distinct keys).  The
 * threshold is found on the device: the radix select's histograms are summed
 * over the parts and the threshold bucket's rows of all parts are ordered
 * together; nothing is copied to the host but the histograms and counts.
 * parts: n_parts distinct contexts created on the same CUDA device with the
 * same n_qubits.  *n_removed (may be NULL): rows removed in all.  Errors:
 * IQCC_ERR_ARG (no, null, repeated or mismatched contexts, NaN eps),
 * IQCC_ERR_OOM, IQCC_ERR_CUDA; IQCC_ERR_STATE when a context is broken.
 */
iqcc_status iqcc_prune_parts(iqcc_ctx* const* parts, int n_parts, double eps, int64_t max_terms,
                             int64_t* n_removed);

/*
 * QMF energy E = sum_k C_k <Omega|P_k|Omega> for the product state of Eq. 3
 * (Eq. 10), theta/phi: host [n_qubits].  <X> = sin(th) cos(ph),
 * <Y> = sin(th) sin(ph), <Z> = cos(th) per qubit.  When every theta_j is
 * exactly 0 or pi (a computational basis state) only strings without X/Y
 * contribute and no sines are evaluated (sin(pi) is taken as 0).
 */
iqcc_status iqcc_qmf_energy(iqcc_ctx* ctx, const double* theta, const double* phi, double* energy);

/*
 * Closed-form energy along one generator: E(tau) = A + B cos(tau) + C sin(tau)
 * for the dressed energy <Omega|e^{-i tau P/2} H e^{i tau P/2}|Omega>
 * (Eq. 5 inserted into Eq. 12).  A: commuting strings; B: anticommuting
 * strings; C: sum over anticommuting T of C_T <i T P>.  abc: host double[3].
 * The minimiser is tau* = atan2(-C, -B); dE/dtau at 0 equals C.
 */
iqcc_status iqcc_generator_abc(iqcc_ctx* ctx, const uint64_t* gx, const uint64_t* gz,
                               const double* theta, const double* phi, double abc[3]);

/*
 * iqcc_generator_abc summed over several contexts (the partitions of one
 * Hamiltonian, App. B: A, B and C are sums over the parts), in part order;
 * with all-zero gx, gz, A is the energy.  tau (may be NULL): the minimiser
 * atan2(-C, -B) of the summed E(tau), 0 when B = C = 0.  Errors as
 * iqcc_generator_abc; IQCC_ERR_ARG also for no or mismatched contexts.
 */
iqcc_status iqcc_generator_abc_parts(iqcc_ctx* const* parts, int n_parts, const uint64_t* gx, const uint64_t* gz,
                                     const double* theta, const double* phi, double abc[3], double* tau);

/*
 * Derivatives of the dressed QMF energy (the adjoint of Eq. 3 / Eq. 12 after
 * Eq. 5), for joint optimisation of the product-state angles and one
 * generator's amplitude.  With a generator (gx, gz: host [W] words each, both
 * non-NULL): *energy = E(tau) = <Omega|e^{-i tau P/2} H e^{i tau P/2}|Omega>
 * = A + B cos(tau) + C sin(tau) as in iqcc_generator_abc, d_theta[j] =
 * dE(tau)/d theta_j and d_phi[j] = dE(tau)/d phi_j (host [n_qubits] each),
 * and *d_tau = -B sin(tau) + C cos(tau).  With gx = gz = NULL: the energy of H
 * and its angle gradient, *d_tau = 0.  H is not modified; the dressed
 * Hamiltonian is never formed.  theta/phi: host [n_qubits]; a qubit whose
 * theta is exactly 0 or pi takes sin(theta) = 0, as in iqcc_qmf_energy.
 * Sums are FP64 with atomic adds, so the last bits can vary between calls.
 * Errors: IQCC_ERR_ARG (NULL output or angle pointer, only one of gx/gz,
 * generator bits above n_qubits), IQCC_ERR_OOM, IQCC_ERR_CUDA.
 */
iqcc_status iqcc_energy_gradients(iqcc_ctx* ctx, const uint64_t* gx, const uint64_t* gz, double tau,
                                  const double* theta, const double* phi, double* energy, double* d_theta,
                                  double* d_phi, double* d_tau);

/*
 * Energy gradients of candidate generators at tau = 0 (Eq. 7 / Eq. 13, sign as
 * above: g = dE/dtau = C of iqcc_generator_abc).
 * n_cand > 0: gradients of the given candidates cx, cz [n_cand][W]; grad[k]
 *   for candidate k (grad: host [n_cand]); ox, oz, cap are ignored and
 *   *n_out = n_cand.
 * n_cand == 0: the Direct Interaction Space of App. A: one candidate per
 *   distinct non-empty flip set F (the x vector) of the terms of H, with Y on
 *   the lowest qubit of F and X on the rest (odd Y count, matching flip set).
 *   When Omega is a basis state (all theta in {0, pi}) only terms with flip
 *   set F contribute (Eq. 14-15): the terms are grouped by flip set in a
 *   partition join (a hash partition of the rows by F, each partition summed
 *   in shared memory); otherwise every term is summed for every candidate
 *   (cost M x G).  Device scratch: 32 bytes (64 when Wd = 4) per term with
 *   a non-empty flip set, and (8 Wd + 8) per candidate.  Candidates are
 *   ordered by |g| with its 20 low mantissa bits cleared (relative tie
 *   tolerance 2^-32), descending, then canonical key ascending.  *n_out = G
 *   (the total); min(cap, G) candidates are written to ox, oz [cap][W] and grad
 *   [cap].  cap = 0 is a size query.
 */
iqcc_status iqcc_dis_gradients(iqcc_ctx* ctx, const double* theta, const double* phi,
                               int64_t n_cand, const uint64_t* cx, const uint64_t* cz,
                               int64_t cap, int64_t* n_out, uint64_t* ox, uint64_t* oz,
                               double* grad);

/* Options and record of one iQCC iteration (App. A procedure steps 1-5). */
typedef struct {
    int n_gen;                 /* generators per iteration (<= 64) */
    double eps;                /* compression threshold, as iqcc_prune */
    int64_t max_terms;         /* term limit, as iqcc_prune (<= 0: none); it holds after every dress */
    double min_gradient;       /* candidates need |g| > this; 0 -> 1e-12 */
    int n_forced;              /* > 0: use these generators instead of screening */
    const uint64_t* forced_x;  /* host [n_forced][W] */
    const uint64_t* forced_z;  /* host [n_forced][W] */
    const double* forced_tau;  /* host [n_forced] or NULL: amplitudes to use */
    int screening;             /* term limit: 0 keeps the largest |C|, 1 the best learned scores
                                  (iqcc_prune_learned with the iteration's generators) */
} iqcc_iter_opts;

typedef struct {
    int n_applied;             /* generators applied */
    uint64_t gx[64 * 4];       /* [n_applied][W] generators, in order */
    uint64_t gz[64 * 4];
    double grad[64];           /* their screening gradients */
    double tau[64];            /* amplitudes used */
    double abc[64][3];         /* A, B, C of each, on the H it dressed */
    int64_t n_terms_before;    /* M at the start of the iteration */
    int64_t n_terms_peak;      /* largest M during the iteration */
    int64_t n_removed;         /* removed by compression */
    int64_t n_terms;           /* M at the end */
    int64_t dressed_terms;     /* sum over generators of M at its dress */
    double energy;             /* QMF energy after compression */
} iqcc_iter_result;

/*
 * One iQCC iteration on the device (App. A steps 1-5; Fig. 1 loop 2a-2c):
 * DIS screening (iqcc_dis_gradients with n_cand = 0) and the top n_gen
 * candidates with |g| > min_gradient (or the forced list); for each in order,
 * A, B, C on the current H, tau = atan2(-C, -B) (0 when B = C = 0; or the
 * forced amplitude), and the dress, after which a Hamiltonian larger than
 * max_terms is cut to the max_terms largest |C| at once (the term limit of the
 * paper's Tables 2-3 holds after every dress, which bounds device memory by
 * 2 max_terms rows); then iqcc_prune(eps, max_terms) and the energy.  The
 * generators of one iteration come from one screening.  A cut is taken as
 * flags and applied by the next dress while it copies H (none after the last
 * dress: the final compression applies the same limit); the A, B, C pass of a
 * generator also counts the rows its dress will keep and bin, so the dress
 * sizes its bins from that count (iqcc_set_bin_slack) and needs no counting
 * pass of its own.
 */
iqcc_status iqcc_iterate(iqcc_ctx* ctx, const double* theta, const double* phi,
                         const iqcc_iter_opts* opts, iqcc_iter_result* out);

/*
 * Device waits.  The stable in-place compaction (the load of canonical
 * input, and a deferred term-limit cut applied outside a dress) waits on other
 * blocks: a tile waits for its predecessors' counts (decoupled look-back); the
 * dress and the compression copy rows out of place and do not wait.  Each
 * wait polls at most
 * `polls` times; then the kernel records IQCC_ERR_TIMEOUT and returns without
 * writing out of bounds, the call that launched it returns IQCC_ERR_TIMEOUT,
 * and the context refuses every later call (IQCC_ERR_STATE).  polls = 0
 * restores the default of 2^24 polls (about a second).  The paper has no
 * counterpart: this bounds every wait of the library.  Errors: IQCC_ERR_ARG.
 */
iqcc_status iqcc_set_wait_limit(iqcc_ctx* ctx, int polls);

/*
 * Self-test of that failure path: one device wait on a word that nothing
 * writes.  Always returns IQCC_ERR_TIMEOUT (after the context's wait limit),
 * and the context then refuses every later call with IQCC_ERR_STATE.  The
 * paper has no counterpart.
 */
iqcc_status iqcc_wait_selftest(iqcc_ctx* ctx);

/* Number of terms currently held. */
iqcc_status iqcc_num_terms(const iqcc_ctx* ctx, int64_t* n_terms);

/*
 * Copy H to the host in canonical order: *n = M; min(cap, M) rows written to
 * x, z [cap][W] and coef [cap].  cap = 0 is a size query.  Rows keep their
 * order through dressing and pruning, so the longest sorted prefix of the
 * table is only merged with the sorted rest.  When x, z and coef are all
 * page-locked host memory registered with CUDA (cudaHostAlloc, a pinned torch
 * tensor) the device writes them directly; other host memory is filled from
 * device scratch with a copy.  Device scratch: about 2 (2 Wd + 1) 8 M bytes.
 */
iqcc_status iqcc_export(iqcc_ctx* ctx, int64_t cap, int64_t* n, uint64_t* x, uint64_t* z,
                        double* coef);

/*
 * As iqcc_export, in the context's storage order (no particular order; each
 * string once): no sort, so the copy runs at the host link's rate.  Meant for
 * moving H out and back in (checkpoints, a host round trip between steps):
 * iqcc_load_hamiltonian accepts rows in any order and sums repeated strings
 * without a sort (or with one, when one string repeats thousands of times).
 * x, z: host [cap][W]; coef: host [cap] (pinned memory copies fastest).
 * Device scratch: 16 W + 8 bytes per row.  A pending term-limit cut of iqcc_iterate is applied
 * first.  Errors: IQCC_ERR_ARG (NULL n, cap < 0, NULL output array with
 * cap > 0), IQCC_ERR_OOM, IQCC_ERR_CUDA.
 */
iqcc_status iqcc_export_rows(iqcc_ctx* ctx, int64_t cap, int64_t* n, uint64_t* x, uint64_t* z, double* coef);

/* Running counters of the context (reset by iqcc_reset_stats). */
typedef struct {
    int64_t n_dress;           /* generators applied */
    int64_t dressed_terms;     /* sum of M over applied generators */
    int64_t anticommuting;     /* sum of anticommuting terms seen */
    int64_t appended;          /* sum of appended terms */
    double dress_kernel_ms;    /* device time of the dress kernels (CUDA events) */
    double dress_bytes;        /* algorithmic bytes of those kernels: 16W M + 16 M_anti + (16W+8) M_new */
    int64_t n_energy;          /* energy / A,B,C passes */
    double energy_kernel_ms;
    double energy_bytes;       /* (16W+8) M per pass */
    double prune_ms;           /* device time of compression */
    double dis_ms;             /* device time of DIS screening */
    double hash_ms;            /* device time of key-index builds (partitioned dress only) */
    int64_t hash_rebuilds;
    int64_t rows_allocated;    /* rows currently allocated on the device */
    int64_t hash_slots;        /* active hash slots */
    int64_t kernel_launches;   /* kernels launched by the library (all contexts) since the reset */
    int64_t n_sorted_groups;   /* generator groups applied by iqcc_dress_sorted */
    double sorted_dress_ms;    /* device time of those groups (expansion, sort, merge; index rebuild excluded) */
    int64_t screen_terms;      /* terms scored by the learned screening perceptron */
    double screen_ms;          /* device time of that scoring (CUDA events) */
    int words;                 /* device words per x or z vector (1, 2 or 4) */
    int pad;
    int64_t fixed_bin_dresses; /* dresses whose bins were sized from the A,B,C pass's count */
    int64_t bin_overflows;     /* of those, dresses redone with exact bins after a bin overflowed */
} iqcc_stats;

iqcc_status iqcc_get_stats(const iqcc_ctx* ctx, iqcc_stats* out);

/*
 * Size of the dress's fixed bins inside iqcc_iterate: a bin holds
 * ceil((1 + frac) * mean) + rows anticommuting rows, mean being the count of
 * the A,B,C pass over the bins (defaults 0.25 and 32: a bin overflows only
 * when the hash spreads far more unevenly than chance allows).  A dress whose
 * bin overflows is redone with exact bins (stats.bin_overflows), so the
 * result does not depend on these values; small ones trade memory for that
 * second pass.  Errors: IQCC_ERR_ARG (frac < 0 or not finite, rows < 0).
 */
iqcc_status iqcc_set_bin_slack(iqcc_ctx* ctx, double frac, int rows);
iqcc_status iqcc_reset_stats(iqcc_ctx* ctx);

/*
 * QMF energy (as iqcc_qmf_energy) of rows the caller already holds in device
 * memory, computed without allocating any device memory.  The paper has no
 * counterpart; it is for callers that cannot allocate when they need the
 * energy: a plug-in whose host framework owns all device memory through its
 * own allocator, a service that must keep a fixed footprint once started.
 *
 * d_rows: device [n_terms][2*Wd] uint64, x words then z words of each string,
 * Wd = 1 (n_qubits <= 64), 2 (<= 128) or 4 (<= 256), words above ceil(n/64)
 * zero; d_coef: device [n_terms] double.  Repeated strings simply add.
 * theta, phi: host [n_qubits]; energy: host double; stream: cudaStream_t or
 * NULL.  Returns after synchronising the stream; the angles are copied from
 * host memory and the result read back, so the call cannot be recorded in a
 * CUDA graph: on a stream that is being captured it returns IQCC_ERR_ARG
 * without issuing any work (the capture stays valid).
 *
 * Scratch is one fixed device array inside the library (234 kB per GPU that
 * loads it, held until the process exits), shared by every call: it limits
 * n_qubits to 256 (larger is IQCC_ERR_ARG with a message) and the energy pass
 * to 4096 blocks.  Calls that overlap on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current.
 * Errors: IQCC_ERR_ARG, IQCC_ERR_CUDA; message in iqcc_last_error(NULL).
 */
iqcc_status iqcc_qmf_energy_noalloc(int n_qubits, int64_t n_terms, const uint64_t* d_rows,
                                    const double* d_coef, const double* theta, const double* phi,
                                    void* stream, double* energy);

/* One-line description of the last error of ctx (or of the calling thread's
   last failed iqcc_load_hamiltonian when ctx is NULL).  Never NULL. */
const char* iqcc_last_error(const iqcc_ctx* ctx);

/* Release the context and all its device memory (NULL is allowed). */
void iqcc_free(iqcc_ctx* ctx);

/* ------------------------------------------------------------------------
 * Partitioned dressing (App. B's bit-wise partitioning, as a data layout).
 * A Hamiltonian may be split over several contexts by the values of chosen
 * key bits: one context per partition, on one GPU or one per GPU.  A
 * generator P that flips none of those bits keeps every pair inside its
 * partition: each context runs iqcc_dress.  A generator that flips some of
 * them pairs every anticommuting row T of partition a with its partner
 * T xor P in partition a xor (P's partition bits); the two contexts then
 * exchange their anticommuting rows (iqcc_cross_rows) and each applies the
 * dress to its own rows with the other's (iqcc_dress_cross).  Energies,
 * A, B, C and DIS gradients are sums over the contexts.
 * ------------------------------------------------------------------------ */

/* Dress two partitions a and b of one Hamiltonian, held by two contexts on
 * the same device, by P at amplitude tau (Eq. 5, library sign) as if they
 * were one context: the anticommuting rows of both go into one set of pair
 * bins (the merge of App. D Eq. 18 as in iqcc_dress), and every output row
 * goes to the partition that owns its key, so a generator that flips the
 * partition bits moves the new partners T xor P to the other context without
 * a copy through the host (App. B's pairwise exchange, on one device).
 * mx, mz: host [W] partition masks; ax, az: host [W], a's bits under them (a
 * key k belongs to a iff k & mask == (ax, az), to b otherwise; every row of
 * a and b must satisfy its side's rule).  All work runs on a's stream; b's
 * stream is synchronised first.  Errors (both unchanged): IQCC_ERR_ARG (same
 * context twice, different devices or qubit counts, bits above n_qubits or
 * outside the masks, non-finite tau), IQCC_ERR_CAPACITY (a context could
 * receive more rows than its capacity: M_a + anticommuting rows of b, and
 * likewise for b), IQCC_ERR_OOM, IQCC_ERR_CUDA; IQCC_ERR_HASH_FULL as
 * iqcc_dress. */
iqcc_status iqcc_dress_pair(iqcc_ctx* a, iqcc_ctx* b, const uint64_t* gx, const uint64_t* gz, double tau,
                            const uint64_t* mx, const uint64_t* mz, const uint64_t* ax, const uint64_t* az);

/* The rows of H that anticommute with P (gx, gz: host [W]): *n = their count;
 * min(cap, *n) of them written to x, z [cap][W] and coef [cap] (host), in no
 * particular order.  cap = 0 is a size query.  H is not changed.  Errors:
 * IQCC_ERR_ARG, IQCC_ERR_OOM, IQCC_ERR_CUDA. */
iqcc_status iqcc_cross_rows(iqcc_ctx* ctx, const uint64_t* gx, const uint64_t* gz, int64_t cap, int64_t* n,
                            uint64_t* x, uint64_t* z, double* coef);

/* Dress H by P at amplitude tau (Eq. 5, library sign) when the partner
 * T xor P of every anticommuting row of H lives in the peer partition, whose
 * anticommuting rows are given (px, pz [n_peer][W], pcoef [n_peer], host,
 * distinct keys; the output of iqcc_cross_rows on the peer).  A local row K
 * that anticommutes becomes C_K cos(tau) + s_T C_T sin(tau) when the peer
 * holds T = K xor P (i T P = s_T P(K)), else C_K cos(tau); each peer row T
 * whose partner K has no local row appends (K, s_T C_T sin(tau)).  With both
 * sides of a pair of partitions called with the other's rows, the union is
 * exactly iqcc_dress on the unsplit Hamiltonian.  Errors (H unchanged):
 * IQCC_ERR_ARG (bad arguments, peer key bits above n_qubits),
 * IQCC_ERR_CAPACITY (M + n_peer rows above capacity), IQCC_ERR_OOM;
 * IQCC_ERR_HASH_FULL, IQCC_ERR_CUDA. */
iqcc_status iqcc_dress_cross(iqcc_ctx* ctx, const uint64_t* gx, const uint64_t* gz, double tau, int64_t n_peer,
                             const uint64_t* px, const uint64_t* pz, const double* pcoef);

/* ------------------------------------------------------------------------
 * Learned term screening (no counterpart in the paper, which limits terms by
 * magnitude).  A perceptron (8 features -> 256 -> 256 -> 1, ReLU, BF16
 * weights and activations with FP32 accumulation on the tensor cores) scores
 * every term from its key and coefficient; the term limit can keep the best
 * scores instead of the largest |C|.  Features of a term T (G = union of the
 * supports of the given generators, <T> at the Eq. 3 reference): log10|C|/8,
 * min(flipped qubits, 16)/16, min(Y letters, 16)/16, Z letters on G/8,
 * |supp T & G|/8, |flips of T & G|/8, <T>, and 1 when every flip of T lies
 * in G (none grows with the number of qubits).  The training
 * target is log10 |C_T E_fut(T)| (iqcc_future_energies): by linearity of the
 * dress, removing T changes the energy after the following generators by
 * exactly -C_T E_fut(T).
 * ------------------------------------------------------------------------ */

/* Weights (host float, row-major): w1 [256][8], b1 [256], w2 [256][256] (row =
 * output unit), b2 [256], w3 [256], b3.  Copied (as BF16 for w1, w2) into the
 * context.  Errors: IQCC_ERR_ARG, IQCC_ERR_OOM, IQCC_ERR_CUDA. */
iqcc_status iqcc_set_screening_model(iqcc_ctx* ctx, const float* w1, const float* b1, const float* w2,
                                     const float* b2, const float* w3, float b3);

/* Features of every term, in the order of iqcc_export: out host float
 * [n_terms][8].  gx, gz: host [n_gen][W] (n_gen <= 64; they define G);
 * theta/phi: host [n_qubits]. */
iqcc_status iqcc_term_features(iqcc_ctx* ctx, int n_gen, const uint64_t* gx, const uint64_t* gz,
                               const double* theta, const double* phi, float* out);

/* E_fut(T) = <Omega| D_k ... D_1 (T) |Omega> of every term T (in the order of
 * iqcc_export): the energy of the single string after the n_gen (<= 8)
 * generators at amplitudes tau (host), expanded along every path as in
 * iqcc_dress_sorted.  out: host double [n_terms]. */
iqcc_status iqcc_future_energies(iqcc_ctx* ctx, int n_gen, const uint64_t* gx, const uint64_t* gz,
                                 const double* tau, const double* theta, const double* phi, double* out);

/* The model's score of every term (in the order of iqcc_export): out host
 * float [n_terms].  Errors: IQCC_ERR_ARG without a model. */
iqcc_status iqcc_term_scores(iqcc_ctx* ctx, int n_gen, const uint64_t* gx, const uint64_t* gz,
                             const double* theta, const double* phi, float* out);

/* The magnitude floor of the learned term limit: frac (in [0, 1], default
 * 0.5) of the limit goes to the largest |C| first, the rest to the best
 * scores among the other terms, so a model that scores badly (outside the
 * sizes it was trained on, say) can never drop the largest terms.  0 ranks
 * every term by its score alone.  Errors: IQCC_ERR_ARG. */
iqcc_status iqcc_set_screening_floor(iqcc_ctx* ctx, double frac);

/* iqcc_prune with the term limit on the model's scores (ties of equal scores
 * in ascending canonical key order) above the magnitude floor; eps still
 * applies to |C|. */
iqcc_status iqcc_prune_learned(iqcc_ctx* ctx, double eps, int64_t max_terms, int n_gen, const uint64_t* gx,
                               const uint64_t* gz, const double* theta, const double* phi, int64_t* n_removed);

/* ------------------------------------------------------------------------
 * Batches of independent Hamiltonians (many small problems screened and
 * dressed together; the paper runs one Hamiltonian at a time, so this has no
 * counterpart there beyond the single-problem steps it repeats).  Each problem
 * has its own qubit count (1..48, one 64-bit word per x and z) and terms; all
 * live in one device context where problem b's strings carry b in z bits
 * 48..63 (Z letters on virtual qubits with theta = 0, which cancel in every
 * product inside a problem and keep problems apart).  References must be
 * z-eigenstates (every theta_j 0 or pi): screening uses the restricted sums of
 * Eq. 14-15.
 * ------------------------------------------------------------------------ */
typedef struct iqcc_batch iqcc_batch;

/* Per-problem results of a screening; every pointer is a host array of B
 * entries (abc: 3 B), all required. */
typedef struct {
    double* energy;     /* E of the problem at the given angles (Eq. 12 at tau = 0) */
    uint64_t* gx;       /* x word of its best DIS candidate (largest |g| as in iqcc_dis_gradients); 0: none */
    uint64_t* gz;       /* z word of that candidate (Y on its lowest flipped qubit) */
    double* grad;       /* the candidate's gradient dE/dtau at 0 (Eq. 7, library sign) */
    double* abc;        /* [B][3] A, B, C of the candidate (iqcc_generator_abc) */
    double* tau;        /* tau* = atan2(-C, -B); 0 without a candidate or when B = C = 0 */
    int64_t* n_terms;   /* terms held by the problem */
} iqcc_batch_screen_out;

/*
 * Load B problems (1..2048): n_qubits[B]; offsets[B + 1] (offsets[0] = 0,
 * non-decreasing) delimit problem b's terms in the host arrays x, z (one word
 * each per term) and coef.  Each problem is canonicalised as by
 * iqcc_load_hamiltonian (repeated strings summed, exact zeros dropped).
 * opts->n_qubits is ignored; capacity, max_probe, stream and the allocator
 * hooks apply to the whole batch.  Errors: IQCC_ERR_ARG (counts, offsets, a
 * qubit count above 48, bits above a problem's qubit count), IQCC_ERR_OOM,
 * IQCC_ERR_CAPACITY, IQCC_ERR_CUDA (message: iqcc_last_error(NULL)).
 */
iqcc_status iqcc_batch_load(iqcc_batch** out, const iqcc_opts* opts, int n_problems, const int* n_qubits,
                            const int64_t* offsets, const uint64_t* x, const uint64_t* z, const double* coef);

/*
 * Screen every problem at its reference (theta/phi: host arrays of the
 * problems' qubit counts concatenated in problem order; theta_j must be 0 or
 * pi): energy, best DIS candidate, its gradient, A, B, C and tau*.  The
 * sequence of kernels runs without host synchronisation; on the first call
 * for a given state of the batch its launch shapes are tuned by timing and it
 * is captured into a CUDA graph, which later calls replay (with the new
 * angles) until a step changes the Hamiltonians.  Errors: IQCC_ERR_ARG (NULL
 * pointer, angles not 0 or pi), IQCC_ERR_HASH_FULL, IQCC_ERR_OOM, IQCC_ERR_CUDA.
 */
iqcc_status iqcc_batch_screen(iqcc_batch* batch, const double* theta, const double* phi,
                              iqcc_batch_screen_out* out);

/*
 * One iteration of every problem with one generator: screen (out as above),
 * dress each problem with its best candidate at its tau* (problems without a
 * candidate are left as they are), remove terms with |C| < eps (eps <= 0:
 * none), then energy_after[B] and n_terms_after[B] (host arrays, may be NULL)
 * at the same angles.  Errors: as iqcc_batch_screen and iqcc_dress.
 */
iqcc_status iqcc_batch_step(iqcc_batch* batch, const double* theta, const double* phi, double eps,
                            iqcc_batch_screen_out* out, double* energy_after, int64_t* n_terms_after);

/* Problem b's terms in canonical order (x, z: host [cap] words, coef [cap]);
 * *n receives the problem's term count.  As iqcc_export. */
iqcc_status iqcc_batch_export(iqcc_batch* batch, int problem, int64_t cap, int64_t* n, uint64_t* x, uint64_t* z,
                              double* coef);

typedef struct {
    int64_t n_terms;        /* terms of all problems */
    int64_t screens;        /* screenings run */
    int64_t graph_replays;  /* of which replays of a captured graph */
    int blocks_energy;      /* tuned grid sizes of the screening kernels */
    int blocks_group;
    int blocks_abc;
    int pad;
} iqcc_batch_info;

iqcc_status iqcc_batch_get_info(const iqcc_batch* batch, iqcc_batch_info* out);
const char* iqcc_batch_last_error(const iqcc_batch* batch);
void iqcc_batch_free(iqcc_batch* batch);

#ifdef __cplusplus
}
#endif

#endif /* IQCC_H */
