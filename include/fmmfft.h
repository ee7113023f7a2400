/*
 * fmmfft.h -- C ABI of the compressed FMM-FFT translation library.
 *
 * The library implements the translation stage of an FMM-FFT matrix-vector
 * product (Qian & Yucel, "On the Compression of Translation Operator Tensors
 * in FMM-FFT-Accelerated SIE Simulators via Tensor Decompositions"):
 *
 *   B_v'(k_p) = IFFT( T~_p . FFT(A_v(k_p)) )                       (Eq. 5)
 *
 * for every plane-wave direction k_p, both field polarisations (theta, phi)
 * and every right-hand side, where T~_p is the FFT'ed translation operator of
 * Eq. 7 on the box-offset grid.  The operators are either stored as they are
 * (format NONE) or compressed at set-up by Tucker, tensor-train (TT) or
 * hierarchical-Tucker (H-Tucker) decompositions in the 3D per-direction or
 * the 4D all-directions format (Sec. II.B, Eqs. 8-14, Algs. 1-3) and restored
 * one direction at a time during the translation (Sec. II.C, Figs. 3-4).
 *
 * Conventions shared by every entry point
 *   - All functions return an int status: FMMFFT_OK (0) or a negative
 *     FMMFFT_ERR_* code.  No C++ exception crosses this interface.
 *   - Complex numbers are interleaved (re, im).  Precision FMMFFT_PREC_C128
 *     uses double pairs (16 bytes); every other precision uses float pairs
 *     (8 bytes).  Host-side import arrays are always double pairs.
 *   - Box grid K = (Kx, Ky, Kz) (the paper's K_x, K_y, K_z, Sec. II.A).  FFT
 *     extents n_i are the smallest powers of two >= 2 K_i - 1 (the circulant
 *     embedding of Sec. II.B; n_i = 2 K_i whenever K_i is a power of two).
 *   - Directions: Gauss-Legendre in cos(theta) (L + 1 nodes, ascending) times
 *     N_phi uniform phi_j = 2 pi j / N_phi, theta-major: p = i * N_phi + j.
 *     N_phi = 2 (L + 1) by default, 2 L + 1 (the paper's N_dir = (L+1)(2L+1),
 *     Sec. II.A) with FMMFFT_KEY_NPHI_RULE = 1.
 *   - Field layout (S_in, S_out): [n_dir][2][nrhs][Kz][Ky][Kx], x fastest,
 *     polarisation 0 = theta, 1 = phi.  One T~_p serves the 2 * nrhs fields
 *     of direction p (Sec. II.A: only the theta and phi components are
 *     translated, with the same scalar operator).
 *   - Operator offsets: offset index d_i = v'_i - v_i in (-K_i, K_i); T~_p is
 *     the unnormalised forward DFT (kernel exp(-2 pi i m k / n)) of the
 *     operator embedded at index d_i mod n_i; near offsets are zero.
 *   - A plan is not thread-safe: calls on one plan must not overlap (its
 *     scratch buffers are shared by all its calls).  Different plans are
 *     independent.
 *   - Device memory for operators and scratch is owned by the plan and freed
 *     by fmmfft_plan_destroy.  Field buffers are owned by the caller.
 */
#ifndef FMMFFT_H_
#define FMMFFT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmmfft_plan_s* fmmfft_plan;
typedef struct fmmfft_batch_s* fmmfft_batch;

/* ---- status codes ------------------------------------------------------ */
enum {
  FMMFFT_OK = 0,
  FMMFFT_ERR_INVALID_ARG = -1,   /* bad size, null pointer, aliasing, ...   */
  FMMFFT_ERR_NOT_COMPRESSED = -2,/* translate before compress / import      */
  FMMFFT_ERR_OOM = -3,           /* device or host allocation failed        */
  FMMFFT_ERR_CUDA = -4,          /* a CUDA runtime call or launch failed    */
  FMMFFT_ERR_UNSUPPORTED = -5,   /* valid request outside this build's limits */
  FMMFFT_ERR_DEVICE = -6,        /* a kernel reported a failure (status word) */
  FMMFFT_ERR_IO = -7,            /* file could not be read or written       */
  FMMFFT_ERR_TOO_LARGE = -8      /* needs more scratch than the fixed buffer of
                                    fmmfft_translate_noalloc holds           */
};

/* ---- storage format and decomposition (Sec. II.B) ---------------------- */
enum {
  FMMFFT_FORMAT_NONE = 0,        /* uncompressed T~_p, n1 x n2 x n3 each    */
  FMMFFT_FORMAT_3D = 3,          /* one decomposition per direction         */
  FMMFFT_FORMAT_4D = 4           /* one decomposition of T_4D (n1,n2,n3,n_dir) */
};
enum {
  FMMFFT_DECOMP_NONE = 0,
  FMMFFT_DECOMP_TUCKER = 1,      /* Eqs. 8-9, Alg. 1                        */
  FMMFFT_DECOMP_TT = 2,          /* Eqs. 13-14, Alg. 3                      */
  FMMFFT_DECOMP_HTUCKER = 3      /* Eq. 11, Alg. 2 (4D format only)         */
};

/* ---- arithmetic of the translation ------------------------------------- */
enum {
  FMMFFT_PREC_C128 = 0,          /* FP64 fields, operators and FFTs          */
  FMMFFT_PREC_C64 = 1,           /* FP32 fields and FFTs, FP32 restores     */
  FMMFFT_PREC_C64_3XTF32 = 2,    /* FP32 fields and FFTs, restores on the tensor
                                    cores as three TF32 products (big x big,
                                    big x small, small x big), FP32 accumulate;
                                    y-z planes of other sides than 32, 64 or
                                    multiples of 64 restore on the CUDA cores */
  FMMFFT_PREC_C64_BF16X3 = 3,    /* as above with bf16 hi/lo splits (hi x hi +
                                    lo x hi + hi x lo, kind::f16 products),
                                    relative error near 2^-16 per product    */
  FMMFFT_PREC_C64_TF32 = 4       /* as 3XTF32 with one TF32 product (operands
                                    rounded to TF32, no split): relative error
                                    near 2^-11 per product, an ablation of the
                                    split modes, coarser than a 1e-4 tolerance */
};

/* ---- keys of fmmfft_plan_set (all before fmmfft_compress) -------------- */
enum {
  FMMFFT_KEY_PRECISION = 1,      /* one of FMMFFT_PREC_* (default C64)          */
  FMMFFT_KEY_NPHI_RULE = 2,      /* 0: N_phi = 2(L+1) (default); 1: 2L+1       */
  FMMFFT_KEY_NEAR_RULE = 3,      /* 0: near iff max|d_i| <= 1 (default);
                                    1: near iff a|d| < kappa * a sqrt(3)/2 (Sec. II.A) */
  FMMFFT_KEY_KAPPA = 4,          /* kappa of near rule 1 (default 4)           */
  FMMFFT_KEY_PREFACTOR = 5,      /* 0: c = 1 (default); 1: c = -k^2 eta/(16 pi^2) (Eq. 7) */
  FMMFFT_KEY_TRUNC_RULE = 6,     /* 0: discarded-energy rule (default);
                                    1: normalised singular value < gamma/sqrt(d) */
  FMMFFT_KEY_PROFILE = 7,        /* 1: record CUDA events between the kernels of
                                    each translation (fmmfft_stage_times); may
                                    be changed at any time                      */
  FMMFFT_KEY_EPS_R_RE = 8,       /* relative permittivity of the medium, real
                                    part (> 0, default 1): k = k0 sqrt(eps_r),
                                    eta = eta0 / sqrt(eps_r) in Eq. 7 (Sec. III.A.5,
                                    Table IV)                                   */
  FMMFFT_KEY_EPS_R_IM = 9,       /* imaginary part (<= 0, default 0; a lossy
                                    medium under the e^{j omega t} convention,
                                    eps_r = eps' - j sigma / (omega eps0))      */
  FMMFFT_KEY_HOST_BLOCKS = 10,   /* direction blocks of fmmfft_translate_host's
                                    copy / compute pipeline (0: default 12; 1:
                                    copy in, translate, copy out in sequence;
                                    at most 64); may be changed at any time   */
  FMMFFT_KEY_DIR_FIRST = 11,     /* shard plans: first direction of the block  */
  FMMFFT_KEY_DIR_COUNT = 12,     /* ... and its length (0, default: through the
                                    last direction of the grid).  A shard plan
                                    holds, compresses and translates only the
                                    directions [first, first + count) of the
                                    grid (Sec. II.A order): n_dir, the
                                    directions, weights and field layouts are
                                    those of the block, so the fields of a
                                    shard are a contiguous block of the whole
                                    problem's.  3D formats and the plain
                                    operator give per direction exactly what
                                    the whole plan gives; 4D formats decompose
                                    the block's own 4D tensor.  Block outside
                                    the grid: INVALID_ARG                     */
  FMMFFT_KEY_RESTORE_ERROR = 13  /* 1: the set-up also measures the FP64
                                    restore error of the stored operator
                                    (fmmfft_stats.restore_rel_err; costs one
                                    host restoration of every direction and a
                                    regeneration of its operator); 0 (default):
                                    not measured                              */
};

/* Stages of one translation, in launch order (fmmfft_stage_times). */
enum {
  FMMFFT_STAGE_RESTORE = 0,      /* restore step 1 of compressed formats      */
  FMMFFT_STAGE_XFWD = 1,         /* forward DFT along x                       */
  FMMFFT_STAGE_YZ = 2,           /* y/z DFTs, Hadamard product, slab restore  */
  FMMFFT_STAGE_XINV = 3,         /* inverse DFT along x                       */
  FMMFFT_NUM_STAGES = 4
};

/* ---- statistics ---------------------------------------------------------- */
typedef struct fmmfft_stats {
  int n_dir;                     /* number of plane-wave directions          */
  int L;                         /* multipole count                          */
  int K[3];                      /* boxes per axis                           */
  int n[3];                      /* FFT extents per axis                     */
  int format, decomp, precision;
  int max_rank[6];               /* largest rank per mode over directions (3D)
                                    or the ranks of the single 4D decomposition;
                                    H-Tucker: r1 r2 r3 r4 r12 r34; TT: r1 r2 r3 */
  double mean_rank[3];           /* mean per-mode rank over directions (3D)   */
  int64_t elements_plain;        /* complex elements of the uncompressed store */
  int64_t elements_compressed;   /* complex elements of the compressed store */
  double saving;                 /* 1 - compressed / plain (Sec. III)        */
  int64_t device_bytes_operator; /* device bytes of the stored operator      */
  int64_t device_bytes_scratch;  /* device bytes of scratch buffers currently held */
  double setup_seconds;          /* wall time of the last fmmfft_compress    */
  int restore_on_tensor_cores;   /* slab restores on the tensor cores (y-z
                                    planes of 32 or 64 per side, or multiples
                                    of 64): 1 in 3xTF32, 2 in BF16x3, 3 in
                                    single TF32; 0 CUDA cores                 */
  int kernel_launches;           /* kernels one fmmfft_translate launches    */
  int large_planes;              /* 1 when the y-z pass keeps restored slabs
                                    in global scratch (planes too large for
                                    shared memory)                           */
  int schedule[4];               /* fmmfft_autotune's choices: x-pass rows per
                                    block multiple (0 = default 2), slab restore
                                    on tensor cores (-1 default, 0 off, 1 on),
                                    pre-pass on tensor cores (same), pre-pass
                                    serial (1) or overlapped (0)            */
  double restore_rel_err;        /* FP64 relative L2 error of the stored
                                    operator's restoration against the plan's
                                    own operator (Eq. 7, embedding, FFT), over
                                    all directions: sqrt(sum_p ||T~_p - R_p||^2
                                    / sum_p ||T~_p||^2), the measure the
                                    tolerance gamma bounds (Algs. 1-3).  Set by
                                    the set-up when FMMFFT_KEY_RESTORE_ERROR is
                                    1: fmmfft_compress, fmmfft_compress_host and
                                    the compressed imports (0 for a plain
                                    operator from fmmfft_compress); -1 when not
                                    measured (also after fmmfft_import_plain and
                                    fmmfft_plan_load)                         */
} fmmfft_stats;

/*
 * Create a plan (host-only; touches no GPU).
 *   Nx, Ny, Nz  boxes per axis, each in [2, 128]        (Sec. II.A, K_x K_y K_z)
 *   a           box edge length (same length unit as 1/k0), > 0
 *   k0          free-space wavenumber, > 0 (2 pi / wavelength); the medium's
 *               permittivity is set with FMMFFT_KEY_EPS_R_RE / _IM
 *   L           multipole count, 0 <= L <= 64            (Sec. II.A)
 *   format      FMMFFT_FORMAT_*; decomp FMMFFT_DECOMP_*; format NONE needs
 *               decomp NONE and vice versa; H-Tucker needs format 4D.
 *   tol         relative tolerance gamma of the decomposition (> 0 unless
 *               decomp is NONE)                           (Algs. 1-3)
 * Errors: FMMFFT_ERR_INVALID_ARG for any violation above, FMMFFT_ERR_OOM.
 */
int fmmfft_plan_create(fmmfft_plan* out, int Nx, int Ny, int Nz, double a, double k0,
                       int L, int format, int decomp, double tol);

/* Set an option (FMMFFT_KEY_*) before fmmfft_compress; INVALID_ARG for an
 * unknown key or value, or when the plan is already compressed. */
int fmmfft_plan_set(fmmfft_plan plan, int key, double value);

/*
 * Set-up on the current CUDA device, blocking: evaluates the translation
 * operator of Eq. 7 in FP64 on the host, embeds and FFTs it (Sec. II.B),
 * decomposes it to tolerance gamma (Algs. 1-3) when decomp != NONE, and
 * uploads the stored form to device memory owned by the plan.
 * Errors: UNSUPPORTED (a size outside this build's kernels), OOM, CUDA.
 */
int fmmfft_compress(fmmfft_plan plan);

/*
 * Load an externally computed uncompressed operator instead of calling
 * fmmfft_compress (format NONE plans only).  That: host array of n_dir * n1 *
 * n2 * n3 complex doubles, index ((p * n1 + x) * n2 + y) * n3 + z, holding
 * T~_p[x][y][z] as defined in the header comment.  Copied; caller keeps it.
 */
int fmmfft_import_plain(fmmfft_plan plan, const double* That);

/*
 * Load externally computed per-direction Tucker factors (format 3D, decomp
 * TUCKER plans only), the representation of Eq. 8 for each direction p:
 *   T~_p[x][y][z] = sum_{a,b,c} C_p[a][b][c] U1_p[x][a] U2_p[y][b] U3_p[z][c].
 * ranks: n_dir * 3 ints (r1, r2, r3 of each direction), each in [1, n_i].
 * core/U1/U2/U3: complex doubles, the directions' arrays concatenated in
 * direction order; C_p is r1 x r2 x r3 (c fastest), U_i_p is n_i x r_i
 * (row-major).  Copied; caller keeps them.
 */
int fmmfft_import_tucker3d(fmmfft_plan plan, const int* ranks, const double* core,
                           const double* U1, const double* U2, const double* U3);

/*
 * Load externally computed per-direction TT factors (format 3D, decomp TT),
 * Eq. 13 for each direction p:
 *   T~_p[x][y][z] = sum_{a,b} U1_p[x][a] C1_p[a][y][b] U3_p[z][b].
 * ranks: n_dir * 2 ints (r1, r2 of each direction).  U1 (n1 x r1), C1
 * (r1 x n2 x r2, last index fastest) and U3 (n3 x r2): complex doubles, the
 * directions' arrays concatenated in direction order.  Copied.
 */
int fmmfft_import_tt3d(fmmfft_plan plan, const int* ranks, const double* U1, const double* C1,
                       const double* U3);

/*
 * Load an externally computed Tucker decomposition of T_4D (format 4D, decomp
 * TUCKER), T_4D[x][y][z][p] = T~_p[x][y][z] (Sec. II.B, Eq. 9):
 *   T_4D[x][y][z][p] = sum C[a][b][c][d] U1[x][a] U2[y][b] U3[z][c] U4[p][d].
 * ranks: 4 ints.  core: r1 x r2 x r3 x r4 (d fastest); U_i: n_i x r_i, U4:
 * n_dir x r4; complex doubles.  Copied.
 */
int fmmfft_import_tucker4d(fmmfft_plan plan, const int* ranks, const double* core, const double* U1,
                           const double* U2, const double* U3, const double* U4);

/*
 * Load an externally computed H-Tucker decomposition of T_4D (format 4D,
 * decomp HTUCKER), balanced tree {1,2},{3,4} (Eq. 11, Alg. 2):
 *   T_4D[x][y][z][p] = sum U1[x][a] U2[y][b] U3[z][c] U4[p][d]
 *                          C12[a][b][s] B[s][t] C34[c][d][t].
 * ranks: 6 ints (r1 r2 r3 r4 r12 r34).  U_i: n_i x r_i (U4: n_dir x r4);
 * C12: r1 x r2 x r12; C34: r3 x r4 x r34; B: r12 x r34; complex doubles,
 * last index fastest.  Copied.
 */
int fmmfft_import_htucker(fmmfft_plan plan, const int* ranks, const double* U1, const double* U2,
                          const double* U3, const double* U4, const double* C12, const double* C34,
                          const double* B);

/*
 * Load an externally computed TT decomposition of T_4D (format 4D, decomp
 * TT), Eq. 14:
 *   T_4D[x][y][z][p] = sum U1[x][a] C1[a][y][b] C2[b][z][c] U3[p][c].
 * ranks: 3 ints (r1 r2 r3).  U1: n1 x r1; C1: r1 x n2 x r2; C2: r2 x n3 x r3;
 * U3: n_dir x r3; complex doubles, last index fastest.  Copied.
 */
int fmmfft_import_tt4d(fmmfft_plan plan, const int* ranks, const double* U1, const double* C1,
                       const double* C2, const double* U3);

/*
 * The translation (Eq. 5) of every field, asynchronous on `stream`
 * (a cudaStream_t; NULL = legacy default stream):
 *   S_out[p][pol][rhs] = crop( IFFT( T~_p . FFT( pad(S_in[p][pol][rhs]) ) ) )
 * restoring T~_p from the stored decomposition when the plan is compressed
 * (Sec. II.C).  S_in, S_out: device pointers, layout and element type as in
 * the header comment, n_dir * 2 * nrhs * Kx * Ky * Kz complex each, must not
 * overlap.  nrhs >= 1.  The first call with a given nrhs (or a larger one than
 * before) allocates the plan's scratch; later calls allocate nothing.
 * Errors: NOT_COMPRESSED, INVALID_ARG, OOM, CUDA (launch failure).  A
 * failure a kernel detects while running (a rank beyond its launch's shared
 * memory, a tensor-core wait that ran out) is not a return value of this
 * asynchronous call: it sets a bit of the plan's status word, which
 * fmmfft_poll_status reads.
 */
int fmmfft_translate(fmmfft_plan plan, const void* S_in, void* S_out, int nrhs, void* stream);

/*
 * Box occupancy (Sec. II.A): boxes that hold no basis function carry no
 * source (A_v = 0) and need no translated field.  `occupied` is a host array
 * of Kx Ky Kz bytes, box index v = (z Ky + y) Kx + x, nonzero for an occupied
 * box; NULL clears the mask (every box occupied, the default).  With a mask,
 * every translation of the plan (fmmfft_translate and its host, batch and
 * allocation-free forms, and fmmfft_translate_disaggregate) reads S_in only
 * at occupied boxes (others taken as zero), writes zero to S_out at empty
 * boxes, and prunes its FFTs: an x-line (y, z) with no occupied box is
 * neither read nor transformed in either x pass.  The result at occupied
 * boxes equals fmmfft_translate of the input with its empty boxes zeroed.
 * May be called before or after fmmfft_compress.  The first call with a mask
 * allocates Kx Ky Kz + Ky Kz bytes on the current device (kept until
 * fmmfft_plan_destroy); every call waits for the device to finish the work
 * already queued (a kernel in flight may read the previous mask) and copies
 * the mask synchronously.  A batch's CUDA graph keeps the occupancy its plans
 * had when it was captured (set masks before a batch's first translation).
 * The mask is not part of plan files.  Errors: INVALID_ARG, OOM, CUDA.
 */
int fmmfft_plan_set_occupancy(fmmfft_plan plan, const unsigned char* occupied);

/*
 * Allocation-free variant of fmmfft_translate (the paper has no counterpart;
 * this is an interface for callers).  Some callers cannot call cudaMalloc
 * while they translate: an iterative solver that runs inside a framework
 * whose memory pool owns the device memory, or a time-critical loop where
 * cudaMalloc / cudaFree would synchronise the device and stall other streams.
 * fmmfft_translate allocates its intermediate buffer on its first call (and
 * again when nrhs grows); this entry point never does.  Its intermediate
 * (the x-transformed fields, n_dir * 2 * nrhs * n1 * Ky * Kz complex) lives in
 * one file-scope device array of FMMFFT_NOALLOC_SCRATCH_BYTES (32 MiB), which
 * every GPU that loads this library holds until the process exits.  The plan's
 * own operator storage, set up by fmmfft_compress or an import, is used as is.
 *
 * Arguments, layouts, ownership and results are those of fmmfft_translate;
 * FMMFFT_KEY_PROFILE is ignored (no stage times are recorded).
 * Set-up: the first call on a device, with that device current, looks up the
 * device address of the array (cudaGetSymbolAddress) and keeps it for the
 * later calls on that device; make that first call before any stream capture
 * begins.  The kept address belongs to the device's current context: after
 * cudaDeviceReset (or anything else that destroys the primary context) it is
 * stale, so do not call this entry point again in that process after a reset.
 * Sharing: every call, from any plan or thread, uses the same array.  Calls
 * whose kernels overlap on the GPU (different streams, or host threads
 * without ordering between them) race on it and give wrong results; order
 * them on one stream.  Nothing needs clearing between calls: the first kernel
 * of a call writes every scratch element that the later ones read.
 * Errors: those of fmmfft_translate except OOM; FMMFFT_ERR_TOO_LARGE (checked
 * before anything is launched) when the intermediate exceeds the array.
 */
#define FMMFFT_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
int fmmfft_translate_noalloc(fmmfft_plan plan, const void* S_in, void* S_out, int nrhs, void* stream);

/*
 * As fmmfft_translate with HOST field buffers: copies S_in to the device,
 * translates and copies the result back, and waits for `stream` before
 * returning.  The directions are taken in FMMFFT_KEY_HOST_BLOCKS blocks
 * (default 12): every block's copy-in is queued on a plan-owned copy stream,
 * block k translates on `stream` once its copy-in is done, and its copy-out
 * runs on a second plan-owned copy stream while block k + 1 translates, so
 * the copies overlap the kernels.  Results equal fmmfft_translate's bit for
 * bit.  Page-locked host buffers are needed for the overlap (pageable ones
 * work, with each copy staged synchronously).  The first pipelined call
 * creates the two copy streams and their events.
 */
int fmmfft_translate_host(fmmfft_plan plan, const void* S_in_host, void* S_out_host,
                          int nrhs, void* stream);

/*
 * Host-only FP64 evaluation of one direction's FFT'ed operator T~_p (Eq. 7,
 * embedded and transformed as in Sec. II.B), exactly as fmmfft_compress
 * computes it, without touching a GPU.  That_out: n1 * n2 * n3 complex
 * doubles, index (x * n2 + y) * n3 + z.  0 <= p < n_dir.
 */
int fmmfft_operator_host(fmmfft_plan plan, int p, double* That_out);

/*
 * Host-only FP64 compression of one direction as fmmfft_compress does it for
 * 3D-format plans (Tucker: Alg. 1), returned restored: ranks_out receives
 * (r1, r2, r3) and restored_out (optional, n1 * n2 * n3 complex doubles,
 * layout as fmmfft_operator_host) the tensor rebuilt from the kept factors.
 * INVALID_ARG for plans of another format; touches no GPU.
 */
int fmmfft_compress_direction_host(fmmfft_plan plan, int p, int* ranks_out, double* restored_out);

/*
 * Host-only FP64 compression of the whole operator exactly as fmmfft_compress
 * does it for the plan's compressed format (Algs. 1-3), restored through the
 * same restore schedule the kernels run (pre-pass products, then the slab
 * formula of each direction), without touching a GPU.  ranks_out: n_dir * 3
 * ints for 3D formats (r1 r2 r3; TT: r1 r2 0), 6 ints for 4D formats (Tucker:
 * r1 r2 r3 r4 0 0; H-Tucker: r1 r2 r3 r4 r12 r34; TT: r1 r2 r3 0 0 0).
 * restored_out (optional): n_dir * n1 * n2 * n3 complex doubles, index
 * ((p * n1 + x) * n2 + y) * n3 + z.  INVALID_ARG for format NONE.
 */
int fmmfft_compress_host(fmmfft_plan plan, int* ranks_out, double* restored_out);
/* On a plan not yet compressed, fmmfft_compress_host also records the
 * statistics of this host compression for fmmfft_plan_stats: ranks,
 * elements_plain / elements_compressed / saving and setup_seconds. */

/*
 * Far-field steps around the translation (Sec. II.A), for the plan's boxes
 * (V = Kx Ky Kz, box index v = (z Ky + y) Kx + x), directions and quadrature
 * weights, with nb basis functions per box (empty slots: zero patterns) and
 * nrhs right-hand sides.  Device arrays, complex64 (complex128 for plans of
 * precision FMMFFT_PREC_C128), interleaved:
 *   patterns  P[p][c][i][v]: theta (c = 0) and phi (c = 1) far-field patterns
 *             P^+(k_p, b_i) of basis function i of box v (Eq. 3), n_dir * 2 *
 *             nb * V elements; P^- is their conjugate;
 *   currents  I[r][i][v]: coefficients of the basis functions, nrhs * nb * V;
 *   A, B      spectra [p][c][r][v] in the layout of fmmfft_translate's S_in /
 *             S_out, n_dir * 2 * nrhs * V;
 *   y         [r][i][v], nrhs * nb * V.
 *
 * fmmfft_aggregate (Eq. 4):    A[p][c][r][v] = sum_i P[p][c][i][v] I[r][i][v]
 * fmmfft_disaggregate (Eq. 6): y[r][i][v] = sum_p w_p sum_c conj(P[p][c][i][v]) B[p][c][r][v]
 *
 * So aggregate -> fmmfft_translate -> disaggregate is the far-field part of the
 * FMM-FFT matrix-vector product (the (-jk/(4 pi)) factor of the Green's
 * function left to the caller).  Asynchronous on `stream`; the plan need not
 * be compressed.  The first call on a plan copies its weights to the current
 * device (8 n_dir bytes, synchronous).  fmmfft_disaggregate sums each
 * output over four consecutive quarters of the directions and adds the four
 * partial sums in a fixed order: results are reproducible bit for bit.
 * Errors: INVALID_ARG (null or misaligned pointers, nb < 1, nrhs outside
 * [1, 4096], an output overlapping an input), UNSUPPORTED (nb > 48), OOM,
 * CUDA (launch failure).
 */
int fmmfft_aggregate(fmmfft_plan plan, const void* patterns, const void* currents, void* A, int nb,
                     int nrhs, void* stream);
int fmmfft_disaggregate(fmmfft_plan plan, const void* patterns, const void* B, void* y, int nb,
                        int nrhs, void* stream);

/*
 * Translation (Eq. 5) and disaggregation (Eq. 6) in one call, the translated
 * fields kept on chip:
 *   y[r][i][v] = sum_p w_p sum_c conj(P[p][c][i][v]) B[p][c][r][v],
 *   B = fmmfft_translate(S_in)
 * with the arrays, layouts and weights of fmmfft_disaggregate.  The inverse x
 * DFT of the translation (the last step of Eq. 5) hands each field's boxes to
 * the sum of Eq. 6 in shared memory, so B is neither stored nor read back.
 * Asynchronous on `stream`; the plan must hold an operator (NOT_COMPRESSED
 * otherwise) and uses its intermediate buffer as fmmfft_translate does
 * (allocated on the first call, or when nrhs grows).  Each output sums over
 * four consecutive quarters of the directions added in a fixed order:
 * reproducible bit for bit (the sum order differs from fmmfft_disaggregate's,
 * so the two agree to rounding).  Errors: those of fmmfft_disaggregate (y
 * must not overlap S_in or the patterns), NOT_COMPRESSED, UNSUPPORTED
 * (Kx > 128, nb > 48).
 */
int fmmfft_translate_disaggregate(fmmfft_plan plan, const void* S_in, const void* patterns, void* y, int nb,
                                  int nrhs, void* stream);

/*
 * The multipole count L of the excess-bandwidth rule (Sec. II.A) for boxes of
 * edge a in a medium of relative permittivity eps_re + j eps_im:
 *   L = floor(x + 1.8 digits^(2/3) x^(1/3)),  x = 2 |k| a sqrt(3)/2,
 *   |k| = k0 |sqrt(eps_r)|,
 * digits the accurate digits of the FMM approximation (the paper's Gamma term
 * read as a digit count).  Host-only.  INVALID_ARG unless a, k0, eps_re,
 * digits > 0 and eps_im <= 0.
 */
int fmmfft_multipole_count(double a, double k0, double eps_re, double eps_im, double digits, int* L_out);

/*
 * Batches of independent translations (many FMM-FFT instances with uneven
 * grids, ranks and RHS counts, Sec. II.C restores per instance).
 *
 * fmmfft_batch_create: a batch over nplans >= 1 existing plans (not copied;
 * they must outlive the batch and be compressed before the first translate).
 * fmmfft_batch_translate: translates instance i from S_in[i] to S_out[i]
 * with nrhs[i] RHS (device pointers and layouts as fmmfft_translate), all
 * asynchronous on `stream`.  The complex64 instances whose y-z planes fit
 * the fused yz kernel (any format and restore arithmetic) run together: they
 * are grouped into shape classes and every phase runs one launch per class
 * for all its instances -- the merged restore pre-pass (one launch per
 * stage), the forward x pass (per x extent), the yz pass (per plane shape,
 * operator kind and restore arithmetic) and the inverse x pass -- whose
 * blocks take the work items of every instance of the class in turn, with
 * the same device code as a single translation, so results equal each
 * instance's fmmfft_translate bit for bit.  Any other
 * instance (complex128, or planes of the large-plane kernel) runs its own
 * launches on one of up to four internal streams.  The environment variable
 * FMMFFT_BATCH_SEPARATE=1 at fmmfft_batch_create gives every instance its
 * own launches.  A device failure inside the shared launches (status word) is
 * reported on the plan whose item raised it, or for the merged pre-pass on
 * the batch's first plan.  When the batch's arguments change, the first call
 * waits for `stream` and uploads the new work descriptors (a few KB).  A
 * call with the same pointers and RHS counts as the previous call is
 * captured as one CUDA graph on its first repetition and replayed from then
 * on (never for the legacy default stream, NULL).  Each plan's intermediate
 * is allocated, if needed, before anything is launched.
 * Errors: those of fmmfft_translate for any instance (nothing of that call is
 * launched when an argument is invalid), CUDA.  A batch is not thread-safe,
 * and its plans must not be translated on their own while a batch call of
 * theirs may still run.
 * fmmfft_batch_destroy: waits for the batch's streams, frees its resources
 * (not the plans).
 */
int fmmfft_batch_create(fmmfft_batch* out, const fmmfft_plan* plans, int nplans);
int fmmfft_batch_translate(fmmfft_batch batch, const void* const* S_in, void* const* S_out,
                           const int* nrhs, void* stream);
int fmmfft_batch_destroy(fmmfft_batch batch);
/* Number of instances that ran in the shared launches of the
 * batch's last fmmfft_batch_translate call (the others ran on their own). */
int fmmfft_batch_shared_count(fmmfft_batch batch, int* count);

/*
 * Autotuner (no counterpart in the paper): times the plan's candidate
 * schedules for `nrhs` RHS with CUDA events on a private stream and applies
 * the fastest.  Candidates: x-pass rows per block (1, 2 or 4 block-line
 * multiples), slab restores and pre-pass products on the tensor cores or the
 * FP32 CUDA cores (3xTF32 plans; the FP32 route is at least as accurate), the
 * pre-pass overlapped with the forward x pass or in line with it.  Stops
 * starting new candidates once budget_ms of wall time has passed (the first
 * always runs).  Allocates and frees two field buffers for the timing.  When
 * the environment variable FMMFFT_TUNE_CACHE names a file, a schedule stored
 * there for the same device, grid, format, precision, ranks and nrhs is
 * applied without timing, and a newly tuned one is appended.  The schedule
 * changes only speed, not the results beyond rounding; fmmfft_stats reports
 * it.  A candidate that sets a bit of the device status word (a rank over its
 * launch's shared memory, a tensor-core wait limit) is dropped; the status
 * word and the stream fmmfft_poll_status waits on are left as the caller's
 * last translation left them (the call first waits for that stream).
 * Errors: NOT_COMPRESSED, INVALID_ARG, OOM, CUDA.
 * fmmfft_batch_autotune: the same for every plan of a batch (nrhs[i] RHS,
 * budget_ms shared evenly); drops the batch's captured graph.
 */
int fmmfft_autotune(fmmfft_plan plan, int nrhs, double budget_ms);
int fmmfft_batch_autotune(fmmfft_batch batch, const int* nrhs, double budget_ms);

/* Fill *out (see fmmfft_stats). */
int fmmfft_plan_stats(fmmfft_plan plan, fmmfft_stats* out);

/* Per-direction ranks of a compressed 3D-format plan: n_dir * 3 ints
 * (r1, r2, r3 of each direction).  INVALID_ARG for other formats or before
 * the plan holds an operator. */
int fmmfft_plan_ranks(fmmfft_plan plan, int* ranks);

/* Unit direction vectors k_p (n_dir x 3 doubles) and quadrature weights w_p
 * (n_dir doubles, summing to 4 pi); either pointer may be NULL. */
int fmmfft_plan_directions(fmmfft_plan plan, double* khat, double* weights);

/* Device milliseconds of each stage (FMMFFT_STAGE_*) of the plan's last
 * translation, from CUDA events recorded on its stream while
 * FMMFFT_KEY_PROFILE was 1 (0 for a stage the format does not run).  Waits for
 * that translation.  INVALID_ARG when no profiled translation has run. */
int fmmfft_stage_times(fmmfft_plan plan, float* ms);

/* Read and clear the plan's device status word (0 = no failure reported).
 * Synchronises the plan's last stream. */
int fmmfft_poll_status(fmmfft_plan plan, int* device_status);

/*
 * Save a plan to a file and load it back (no counterpart in the paper: the
 * FP64 set-up of the 4D formats takes minutes, a load seconds).  The file
 * holds the plan's parameters and options and, for compressed plans, the
 * stored factors (in FP64) with their restore schedule; plain plans are
 * regenerated on load.  fmmfft_plan_save needs a compressed (ready) plan;
 * fmmfft_plan_load creates a ready plan on the current device (*out, to be
 * destroyed by the caller).  Errors: IO (file cannot be opened, read or
 * written), INVALID_ARG (not a plan file of this version, or inconsistent
 * contents), and those of fmmfft_compress on load.
 */
int fmmfft_plan_save(fmmfft_plan plan, const char* path);
int fmmfft_plan_load(fmmfft_plan* out, const char* path);

/* Release every resource of the plan (device memory included). */
int fmmfft_plan_destroy(fmmfft_plan plan);

/* Static text for a status code. */
const char* fmmfft_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* FMMFFT_H_ */
