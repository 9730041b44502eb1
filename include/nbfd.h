/*
 * nbfd.h -- C ABI of libnbfd, a GB300 (sm_103a) decoder for (2,k)-regular non-binary LDPC
 * codes over GF(2^m) using the Log-Fourier sum-product algorithm of Kasai & Sakaniwa,
 * "Fourier Domain Decoding Algorithm of Non-Binary LDPC Codes for Parallel Implementation",
 * IEICE Trans. Fundamentals 93(11), 2010.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - q = 2^m, 2 <= m <= 8. A field element is an integer in [0, q): bit i-1 is the coefficient
 *   of alpha^(i-1) (Section 2, m-bit representation).
 * - Edges are held in check-major order: library edge slot e = c*k + j is the j-th edge of
 *   check c. nbfd_code_edge_order() maps slots back to the caller's edge indices.
 * - Message vectors ("Gamma form", Section 3.2): one float32 per z in GF(2^m), laid out
 *   [frame][edge][z] (or [frame][variable][z]), contiguous in z. The float's sign bit is the
 *   GF(2) sign of P(z); its magnitude is -ln|P(z)| >= 0 (+inf when P(z) = 0). Every message the
 *   library writes is normalised so that P(0) = 1 (stored as +0.0f).
 * - Channel input: bit LLRs L = ln Pr(b=0|y)/Pr(b=1|y), float32 laid out [frame][variable][bit],
 *   bit i-1 <-> coordinate of alpha^(i-1).
 * - Pointers named *_dev are device pointers on the device current when the code was created;
 *   the caller owns them and the library never frees them. Work is enqueued on `cuda_stream`
 *   (a cudaStream_t; NULL = legacy default stream).
 * - Every call returns an int status (NBFD_OK = 0 or a negative NBFD_E* code) and never throws;
 *   nbfd_last_error() gives a message for the calling thread's last failure.
 */
#ifndef NBFD_H
#define NBFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------- */
#define NBFD_OK 0
#define NBFD_EINVAL (-1)    /* bad argument (null pointer, size out of range, ...) */
#define NBFD_ENOTREG (-2)   /* graph is not (2,k)-regular, or counts disagree */
#define NBFD_EPOLY (-3)     /* polynomial not of degree m, or not primitive */
#define NBFD_EDUP (-4)      /* a (check, variable) pair appears twice */
#define NBFD_EZERO (-5)     /* an edge entry h_cv is 0 or >= q */
#define NBFD_ENOMEM (-6)    /* host or device allocation failed / workspace too small */
#define NBFD_ECUDA (-7)     /* a CUDA runtime call failed (message in nbfd_last_error) */
#define NBFD_ETIMEDOUT (-8) /* a bounded device-side wait gave up */
#define NBFD_EBUSY (-9)     /* over budget: retry later */
#define NBFD_ENOTSUP (-10)  /* form / size not supported by this build */

/* ---- variable-node convolution forms (Section 3.2, the boxplus definition) ----------- */
#define NBFD_FORM_FP32_DIRECT 0 /* q^2-term signed sum of exponentials per output, FP32 */
#define NBFD_FORM_BF16_HGEMM 1  /* Hadamard transforms on tensor cores, BF16 in / FP32 acc */
#define NBFD_FORM_FP16_HGEMM 2  /* same, FP16 in / FP32 acc */
#define NBFD_FORM_FP32_FWHT 3   /* fast Walsh-Hadamard butterflies, FP32 */
#define NBFD_FORM_FP32_TC 4     /* Hadamard transforms on tensor cores, operands split into three
                                   bf16 parts (24 bits) with FP32 accumulate */
#define NBFD_FORM_FP64_DIRECT 5 /* the direct form with the variable node's sums in FP64 (the
                                   Section 3.2 convolution step run in FP64; messages stay FP32) */
/* The tensor-core forms (1, 2, 4) need m = 8 (q = 256 = 16 x 16); other m give NBFD_ENOTSUP. */
/* Decision flag, OR'ed into a form: the tentative symbol is argmax_x mu_v(x), the symbol-MAP form
 * of Section 3.2 (mu_v = inverse transform of M_v, taken directly from the x-domain product),
 * instead of the bitwise read-out of M_v(alpha^{i-1}); the stop test then uses the GF(2^m)
 * syndrome alone (the Fourier-domain syndrome describes bitwise decisions). Ties go to the lowest
 * symbol. Supported with the FWHT and tensor-core forms (not with NBFD_FORM_FP32_DIRECT). */
#define NBFD_DECIDE_SYMBOL 0x100
/* Storage flag, OR'ed into a form: messages kept in device memory as IEEE half instead of
 * float -- the same Gamma word (sign bit = GF(2) sign, value = -ln|P|) with its log-magnitude
 * rounded to an 11-bit significand; all arithmetic stays FP32. Halves the bytes every iteration
 * moves (the low-precision message storage the paper's log domain allows, Section 3.2). Message
 * buffers of nbfd_var_update and the *_f16 step calls are then uint16 [frame][slot][z].
 * Error added per stored entry: |d ln|P|| <= 2^-11 |ln|P||, i.e. |dP| <= 2^-11 / e. Supported
 * with NBFD_FORM_FP32_FWHT at m = 8 (other combinations give NBFD_ENOTSUP); not by the server. */
#define NBFD_STORE_F16 0x200
/* Path flag, OR'ed into a form: decode GF(16) codes with the per-iteration kernels (one check,
 * variable-node and stop launch per iteration over every active frame) even where the fused
 * small-code kernel applies. Without it, nbfd_decode and nbfd_decode_batch decode the frames of a
 * GF(16) code whose per-frame messages fit in shared memory (the FWHT form, float storage) in one
 * launch that keeps each frame on chip for all of its iterations; both paths give bit-identical
 * outputs. The paper has no counterpart (it is a choice of schedule, not of arithmetic). */
#define NBFD_UNFUSED 0x400
/* Path flags for the tensor-core forms (NBFD_FORM_BF16_HGEMM, _FP16_HGEMM, _FP32_TC): the
 * Hadamard products as tcgen05 MMAs (operands staged in shared memory, FP32 accumulators in tensor
 * memory, 8 variables' 16 x 16 blocks stacked into M = 128; NBFD_TCGEN05) or as warp-level
 * mma.sync m16n8k16 (NBFD_MMA_SYNC). Same operand precision, FP32 accumulation either way.
 * Without a flag each form takes the path measured faster on GB300: tcgen05 for
 * NBFD_FORM_FP32_TC (three operand parts per product), mma.sync for the BF16 / FP16 forms. Both
 * flags, or either with another form: NBFD_ENOTSUP. The paper has no counterpart. */
#define NBFD_TCGEN05 0x800
#define NBFD_MMA_SYNC 0x1000

typedef struct nbfd_code nbfd_code; /* opaque, library-owned, immutable after creation */

/*
 * nbfd_code_create -- load a (2,k)-regular code H = {h_cv} (Section 2: M x N over GF(2^m),
 * column weight j = 2, row weight k, M = 2N/k).
 *   N, M, k, m       : sizes; requires 2 <= m <= 8, 2 <= k <= 32, n_edges == 2N == M*k.
 *   prim_poly        : primitive polynomial of alpha, bit j = coefficient of x^j (e.g. 0x11D).
 *   edge_check/var/h : host arrays of n_edges entries, in any order: the edge (c, v) carries
 *                      h_cv in [1, q). Copied; the caller keeps ownership.
 *   out              : receives the handle (device tables are allocated on the current device).
 * Errors: NBFD_EINVAL, NBFD_ENOTREG, NBFD_EPOLY, NBFD_EDUP, NBFD_EZERO, NBFD_ENOMEM, NBFD_ECUDA.
 */
int nbfd_code_create(int N, int M, int k, int m, uint32_t prim_poly, int n_edges,
                     const int32_t *edge_check, const int32_t *edge_var, const uint16_t *edge_h,
                     nbfd_code **out);

/* Free a handle (NULL is ignored). No decode using it may be in flight. */
void nbfd_code_destroy(nbfd_code *code);

/* Sizes of a handle (any out pointer may be NULL). */
int nbfd_code_info(const nbfd_code *code, int *N, int *M, int *k, int *m);

/* caller_edge_of_slot[e] (host, n_edges entries) = index in the caller's edge arrays of library
 * edge slot e (check-major order). */
int nbfd_code_edge_order(const nbfd_code *code, int32_t *caller_edge_of_slot);

/*
 * nbfd_field_index_map -- host-only (no device work): the Fourier index map of GF(2^m) for the
 * primitive polynomial prim_poly, table[h*q + z] = H z with H = (A^i)^T for h = alpha^i
 * (Section 3.1 check-to-variable step; Appendix A). Row h = 0 is zero. `table` holds q*q bytes.
 * Errors: NBFD_EINVAL (m outside [2, 8] or table NULL), NBFD_EPOLY.
 */
int nbfd_field_index_map(int m, uint32_t prim_poly, uint8_t *table);

/* Host copy of the Fourier index map of Section 3.1 / Appendix A: table[h*q + z] = H z with
 * H = (A^i)^T for h = alpha^i (row h = 0 is zero). `table` holds q*q bytes. */
int nbfd_code_index_map(const nbfd_code *code, uint8_t *table);

/*
 * nbfd_decode_workspace_size -- bytes of device scratch that nbfd_decode needs for n_frames
 * frames, max_iter iterations and the given form (messages in both directions, per-edge
 * syndrome words, active-frame lists and counters).
 */
size_t nbfd_decode_workspace_size(const nbfd_code *code, int n_frames, int max_iter, int form);

/*
 * nbfd_decode -- full decoder of Section 2 (INITIALIZATION, then CHECK TO VARIABLE, VARIABLE TO
 * CHECK and TENTATIVE DECISION repeated) with the Log-Fourier rules of Section 3.2:
 *   INIT   Lambda0 = Gamma(WHT(p0)) from the bit LLRs, sent on both edges of every variable;
 *   C->V   permute by H_cv, leave-one-out sum over the other k-1 edges, permute by H_cv^{-1};
 *   V->C   Lambda0 [+] Lambda_c'v (boxplus log-convolution), normalised to P(0) = 1;
 *   TENT.  bit i of x_hat_v = sign of M_v(alpha^{i-1}); Fourier syndrome bit i of check c =
 *          XOR over V_c of the signs of M_v(H_cv alpha^{i-1}).
 * A frame stops at iteration l (1 <= l <= max_iter) when all its Fourier syndrome bits are 0
 * and the GF(2^m) syndrome of x_hat is 0; stopped frames are dropped from later iterations.
 *   n_frames        : F >= 0 (F = 0 returns NBFD_OK without work).
 *   llr_dev         : [F][N][m] float32 bit LLRs (device).
 *   max_iter        : >= 1.
 *   form            : NBFD_FORM_*.
 *   symbols_dev     : [F][N] uint16 out: the last tentative decision of each frame.
 *   syndrome_ok_dev : [F] uint8 out: 1 iff H x_hat = 0 for the output symbols.
 *   iters_dev       : [F] int32 out: iteration at which the frame stopped (max_iter if never).
 *   workspace_dev   : device scratch of >= nbfd_decode_workspace_size() bytes, 256-byte
 *                     aligned; NULL makes the call allocate and free it on `cuda_stream`.
 * The call is stream-ordered but synchronises with `cuda_stream` every few iterations to test
 * for early termination (it returns after the last iteration's kernels completed).
 * Errors: NBFD_EINVAL, NBFD_ENOTSUP, NBFD_ENOMEM, NBFD_ECUDA.
 */
int nbfd_decode(const nbfd_code *code, int n_frames, const float *llr_dev, int max_iter, int form,
                uint16_t *symbols_dev, uint8_t *syndrome_ok_dev, int32_t *iters_dev,
                void *workspace_dev, size_t workspace_bytes, void *cuda_stream);

/* ---- uneven batches ------------------------------------------------------------------------
 * Frames of several codes (different N, k and q) decoded by one call: the same algorithm as
 * nbfd_decode (Sections 2 and 3.2, the same stop rule and outputs) for every code. The
 * iteration loop runs as a CUDA graph replayed by the host: one graph holds two iterations of
 * every code, each code a separate branch, and the loop state (active-frame lists and counts,
 * iteration number) lives in device memory, so the graph needs no per-iteration arguments.
 * The host reads the active counts every few replays and stops when no frame is left or
 * max_iter iterations have run. */

#define NBFD_BATCH_AUTOTUNE 1 /* flags: time launch shapes for shapes not tuned yet (see below) */

/* Device scratch for nbfd_decode_batch (0 on a bad argument). */
size_t nbfd_decode_batch_workspace_size(int n_codes, const nbfd_code *const *codes,
                                        const int *n_frames, int max_iter, int form);

/*
 * nbfd_decode_batch -- decode n_codes groups of frames; group i has n_frames[i] >= 0 frames of
 * codes[i] (every code on the current device; 1 <= n_codes <= 64).
 *   llr_dev[i]     : [n_frames[i]][N_i][m_i] float32 bit LLRs (device).
 *   form           : NBFD_FORM_* (+ NBFD_DECIDE_SYMBOL), supported by every code's field.
 *   flags          : 0 or NBFD_BATCH_AUTOTUNE.
 *   symbols_dev[i], syndrome_ok_dev[i], iters_dev[i] : outputs of group i as in nbfd_decode.
 *   workspace_dev  : >= nbfd_decode_batch_workspace_size() bytes, 256-byte aligned, or NULL
 *                    (allocated and freed on `cuda_stream`).
 * Returns after the last iteration's kernels completed. Errors: NBFD_EINVAL, NBFD_ENOTSUP,
 * NBFD_ENOMEM, NBFD_ECUDA, NBFD_ETIMEDOUT.
 */
int nbfd_decode_batch(int n_codes, const nbfd_code *const *codes, const int *n_frames,
                      const float *const *llr_dev, int max_iter, int form, int flags,
                      uint16_t *const *symbols_dev, uint8_t *const *syndrome_ok_dev,
                      int32_t *const *iters_dev, void *workspace_dev, size_t workspace_bytes,
                      void *cuda_stream);

/*
 * nbfd_autotune -- time candidate launch shapes of the check kernel (warps per block, bulk-copy
 * pipeline depth, blocks per SM; for q >= 128 also its team variant) and of the variable-node
 * kernel (blocks per SM; warps per block
 * for GF(64)) for this code,
 * n_frames and form, on scratch buffers it allocates on `cuda_stream`, and keep the fastest.
 * Later nbfd_decode / nbfd_decode_batch calls with the same device, code shape (N, k, m),
 * n_frames and form use it. Synchronises `cuda_stream`. The paper has no counterpart.
 * Errors: NBFD_EINVAL, NBFD_ENOTSUP, NBFD_ECUDA.
 */
int nbfd_autotune(const nbfd_code *code, int n_frames, int form, void *cuda_stream);

/* The shape nbfd_autotune chose (NBFD_EINVAL if this shape was never tuned). check_warps < 0:
 * the check kernel's team variant, where the -check_warps warps of a block share one pipeline of
 * whole checks (q >= 128; check_stages is then per block). var_warps: warps per block of the
 * variable-node kernel where it has several block shapes (GF(64): 4, 7 or 15), 0 where it has
 * one. Any out pointer may be NULL. */
int nbfd_autotune_result(const nbfd_code *code, int n_frames, int form, int *check_warps,
                         int *check_stages, int *check_blocks_per_sm, int *var_blocks_per_sm,
                         int *var_warps);

/*
 * nbfd_last_decode_stats -- for the calling thread's last successful nbfd_decode or
 * nbfd_decode_noalloc: the number of (frame, iteration) pairs where the Fourier-domain syndrome
 * of Section 3.2 cleared while the GF(2^m) syndrome H x_hat was not 0 (the frame went on
 * decoding: the stop test needs both).
 * Errors: NBFD_EINVAL (NULL pointer, or no such call in this thread).
 */
int nbfd_last_decode_stats(long long *fourier_only_clears);

/* ---- decoding without device allocation ----------------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers of the library. */

/* Size of the fixed scratch array behind nbfd_decode_noalloc (64 MiB). */
#define NBFD_NOALLOC_SCRATCH_BYTES (64ull << 20)

/*
 * nbfd_decode_noalloc -- the same decoding as nbfd_decode (the same loop, launch shapes and
 * synchronisation with `cuda_stream`: the host reads the active-frame count back every few
 * iterations; the same outputs, status codes -- NBFD_ETIMEDOUT when a bounded device-side wait
 * expired -- and nbfd_last_decode_stats), for callers that must not allocate device memory while
 * decoding: a receiver whose device memory another runtime reserved up front, or a real-time loop
 * where cudaMalloc/cudaFree are banned because they may synchronise the device and take
 * unbounded time. It calls no allocating routine (host reads go to pageable words on the stack;
 * nbfd_prof_enable's timers are not used).
 *   - Its scratch is a fixed NBFD_NOALLOC_SCRATCH_BYTES array inside the library, created when the
 *     library's device code is loaded on a device and held on every such device until the
 *     process exits.
 *   - The first call on each device looks the array's address up (with that device current);
 *     make that first call before any stream capture.
 *   - A batch whose scratch (nbfd_decode_workspace_size) exceeds the array is rejected with
 *     NBFD_ENOMEM and a message; split it into smaller calls. At GF(256), N = 512 and
 *     max_iter <= 100 that is up to 31 frames per call (62 with NBFD_STORE_F16).
 *   - Every call uses the same array and clears what it needs at its start. Calls whose GPU work
 *     can overlap (different streams without ordering between them, or several host threads)
 *     race on the array and corrupt each other's results: order them.
 */
int nbfd_decode_noalloc(const nbfd_code *code, int n_frames, const float *llr_dev, int max_iter,
                        int form, uint16_t *symbols_dev, uint8_t *syndrome_ok_dev,
                        int32_t *iters_dev, void *cuda_stream);

/* ---- step-level entry points (one step of Section 3.2 each, all frames, no early stop) -- */

/*
 * nbfd_init_messages -- INITIALIZATION of Section 3.2: p0_v(x) = prod_i Pr(b_i = x_i | y_i),
 * P0_v = WHT(p0_v) (Section 2.1 definition, computed with butterflies), Lambda0_v = Gamma(P0_v)
 * normalised to P0(0) = 1.
 *   llr_dev     : [F][N][m] float32.
 *   lambda0_dev : [F][N][q] float32 Gamma form out, or NULL.
 *   v2c_dev     : [F][E][q] float32 out (Lambda0 of each slot's variable), or NULL.
 */
int nbfd_init_messages(const nbfd_code *code, int n_frames, const float *llr_dev,
                       float *lambda0_dev, float *v2c_dev, void *cuda_stream);

/*
 * nbfd_check_update -- CHECK TO VARIABLE of Section 3.2 for every check of every frame:
 * Lambda~_vc(z) = Lambda_vc(H_cv z); Lambda~_cv = Gamma-sum over the other k-1 edges (signs XOR,
 * log-magnitudes add, computed without subtraction so +inf entries stay exact);
 * Lambda_cv(z) = Lambda~_cv(H_cv^{-1} z).
 *   v2c_dev : [F][E][q] in; c2v_dev : [F][E][q] out (must not alias v2c_dev).
 */
int nbfd_check_update(const nbfd_code *code, int n_frames, const float *v2c_dev, float *c2v_dev,
                      void *cuda_stream);

/*
 * nbfd_var_update -- VARIABLE TO CHECK and TENTATIVE DECISION of Section 3.2 for every
 * variable of every frame. The channel message Lambda0_v is recomputed from the LLRs with the
 * same device code as nbfd_init_messages (it is not read from memory).
 *   V->C: Lambda_vc = Lambda0_v [+] Lambda_c'v (c' the other check of v), normalised.
 *   M_v  = Lambda0_v [+] Lambda_c1v [+] Lambda_c2v, evaluated at the 3m points it is needed at.
 *   llr_dev      : [F][N][m] in.      c2v_dev : [F][E][q] in.
 *   v2c_dev      : [F][E][q] out (must not alias c2v_dev).
 *   symbols_dev  : [F][N] uint16 out, bit i-1 = sign bit of M_v(alpha^{i-1}) (or NULL).
 *   fsyn_dev     : [F][E] uint8 out, bit i-1 = sign bit of M_v(H_cv alpha^{i-1}) for the edge's
 *                  (c, v) (or NULL).
 */
int nbfd_var_update(const nbfd_code *code, int n_frames, int form, const float *llr_dev,
                    const float *c2v_dev, float *v2c_dev, uint16_t *symbols_dev, uint8_t *fsyn_dev,
                    void *cuda_stream);

/* INITIALIZATION and CHECK TO VARIABLE with half-precision message storage (NBFD_STORE_F16):
 * as nbfd_init_messages (without lambda0) and nbfd_check_update, with uint16 message buffers
 * [F][E][q] holding IEEE halves. Errors as those calls; NBFD_ENOTSUP unless m = 8. */
int nbfd_init_messages_f16(const nbfd_code *code, int n_frames, const float *llr_dev,
                           uint16_t *v2c_dev, void *cuda_stream);
int nbfd_check_update_f16(const nbfd_code *code, int n_frames, const uint16_t *v2c_dev,
                          uint16_t *c2v_dev, void *cuda_stream);

/*
 * nbfd_syndrome -- syndromes of Section 3.1/3.2 for every check of every frame:
 *   fourier_dev[f][c] = XOR over the k edges of c of fsyn_dev[f][e]  (Fourier-domain syndrome);
 *   exact_dev[f][c]   = sum_{v in V_c} h_cv x_v over GF(2^m)          (x = symbols_dev[f]).
 *   symbols_dev : [F][N] uint16 in; fsyn_dev : [F][E] uint8 in (may be NULL: fourier not
 *   written); fourier_dev, exact_dev : [F][M] uint16 out (either may be NULL).
 */
int nbfd_syndrome(const nbfd_code *code, int n_frames, const uint16_t *symbols_dev,
                  const uint8_t *fsyn_dev, uint16_t *fourier_dev, uint16_t *exact_dev,
                  void *cuda_stream);

/* ---- serving: continuous batching of single-frame requests ----------------------------
 * The decoding of Section 2 / Section 3.2 applied to a stream of requests: a worker thread keeps
 * one pool of resident frame slots per code (messages of both directions stay in device memory
 * across iterations), admits queued requests into free slots between rounds, runs one decoding
 * iteration per round over every pool (pools on separate streams overlap on the device), and
 * retires each frame as soon as its Fourier-domain and GF(2^m) syndromes are zero or its own
 * max_iter is reached. A frame's result does not depend on the other frames in flight. */
typedef struct nbfd_server nbfd_server;

/* Start a server on the current device. mem_budget_bytes bounds the device memory of all pools
 * (a pool is sized from what is left when its code is first registered or submitted, at most
 * 4096 slots); form is an NBFD_FORM_* for every request. */
int nbfd_srv_create(size_t mem_budget_bytes, int form, nbfd_server **out);

/* Create the pool of a code now rather than at its first submission: its device memory, streams
 * and pinned staging buffers are allocated here, so that the first requests do not wait for
 * them. Registering a code twice is a no-op. Errors as nbfd_srv_submit. */
int nbfd_srv_register(nbfd_server *srv, const nbfd_code *code);

/* Queue one frame: llr_host [N][m] float32 (copied), max_iter >= 1. *ticket identifies it.
 * NBFD_EBUSY: no pool fits the remaining budget or the queue is full -- retry later.
 * NBFD_ENOTSUP: the server's form does not support this code's m. */
int nbfd_srv_submit(nbfd_server *srv, const nbfd_code *code, const float *llr_host, int max_iter,
                    uint64_t *ticket);

/* Returns 1 and fills the outputs (symbols_host [N] uint16, *ok, *iters, *latency_s = seconds
 * from submit to retirement; any may be NULL) once the ticket's frame retired, 0 while it is
 * queued or in flight, < 0 for an unknown ticket or a server error. A ticket is reported once. */
int nbfd_srv_poll(nbfd_server *srv, uint64_t ticket, uint16_t *symbols_host, uint8_t *ok,
                  int32_t *iters, double *latency_s);

/* Seconds on the server's monotonic clock (the clock latencies are measured on). */
double nbfd_srv_clock(void);

/* Queue n frames of one code at once: llr_host [n][N][m]; arrival (may be NULL) gives each
 * frame's arrival time on nbfd_srv_clock() -- latency is then measured from it; tickets [n] out.
 * All n tickets and the queue room are taken before any frame is copied; the frames are then
 * copied and queued in chunks, so the worker may start on the first frames before the call
 * returns. Errors as nbfd_srv_submit (no frame is queued on error). */
int nbfd_srv_submit_many(nbfd_server *srv, const nbfd_code *code, int n, const float *llr_host,
                         int max_iter, const double *arrival, uint64_t *tickets);

/* Take up to max_n retired frames in retirement order: tickets, flags, iteration counts and
 * latencies (any array may be NULL). Returns how many were taken (0 if none), < 0 on a server
 * error. Frames taken here are no longer reported by nbfd_srv_poll. */
int nbfd_srv_collect(nbfd_server *srv, int max_n, uint64_t *tickets, uint8_t *ok, int32_t *iters,
                     double *latency_s);

/* Rounds run so far, frames queued and in flight, device bytes held by pools. */
int nbfd_srv_stats(nbfd_server *srv, long long *rounds, long long *queued, long long *in_flight,
                   size_t *device_bytes);

/* Cumulative wall seconds the worker thread has spent in each phase since the server started:
 * seconds[0] admission (moving queued frames into free slots and staging their LLRs in pinned
 * memory), [1] issuing rounds (launches and copies), [2] waiting for the oldest round on the
 * device, [3] retiring (result copies, ticket completion), [4] idle (no work). seconds [5] out. */
int nbfd_srv_worker_times(nbfd_server *srv, double *seconds);

/* Stop the worker and free the pools (pending requests are dropped). No other call on srv may
 * run concurrently with this one. */
void nbfd_srv_destroy(nbfd_server *srv);

/* ---- kernel timers (CUDA events around every launch of nbfd_decode) -------------------- */
#define NBFD_KERNEL_INIT 0
#define NBFD_KERNEL_CHECK 1
#define NBFD_KERNEL_VAR 2
#define NBFD_KERNEL_SYNDROME 3
#define NBFD_KERNEL_TAIL 4 /* the remaining iterations of the last few frames, one launch */
#define NBFD_KERNEL_FUSED 5 /* whole decodes of small GF(16) codes, one launch */
#define NBFD_KERNEL_COUNT 6

/* Time the kernels whose bit (1 << NBFD_KERNEL_*) is set in kernel_mask (0 disables; NBFD_PROF_ALL
 * times all six) for the calling process; resets the totals. Each timed launch adds two event
 * records to the stream. */
#define NBFD_PROF_ALL 0x3F
int nbfd_prof_enable(int kernel_mask);
/* Totals since the last enable: device milliseconds, launches, and frame-units (the sum over
 * launches of the number of frames the launch processed). Any out pointer may be NULL. */
int nbfd_prof_get(int kernel, double *ms, long long *launches, long long *frame_units);

/* ---- conventional Log-SP (Section 2.2), the decoder Log-Fourier SP reformulates ------------
 * Kept to measure Table 1 on the GPU: its check node carries the log-convolutions, its variable
 * node only component-wise additions. Messages are x-domain log-probabilities lambda(x) in
 * [-inf, 0] as float32 (no sign bit), [F][slot][x] with the check-major slots of the code; m in
 * [3, 8]. No decoding loop: the calls are one step each over every frame, like the step-level
 * calls above. Errors: NBFD_EINVAL, NBFD_ENOTSUP, NBFD_ECUDA. */

/* INITIALIZATION: lambda_vc = lambda0_v(x) = ln Pr(X_v = x | y_v) = sum_i ln Pr(b_i = x_i | L_i)
 * on both edges of every variable. llr_dev [F][N][m] in, v2c_dev [F][E][q] out. */
int nbfd_logsp_init(const nbfd_code *code, int n_frames, const float *llr_dev, float *v2c_dev,
                    void *cuda_stream);

/* CHECK TO VARIABLE (the log-convolution of Section 2.2): lambda~_vc(x) = lambda_vc(h^{-1} x);
 * lambda~_cv = the log-convolution of the other k - 1 lambda~_v'c (computed as linear XOR
 * convolutions of their max-shifted exponentials, prefix and suffix products); lambda_cv(x) =
 * lambda~_cv(h x), normalised to max_x lambda_cv(x) = 0. Needs k >= 3. v2c_dev in, c2v_dev out
 * ([F][E][q], must not alias). */
int nbfd_logsp_check_update(const nbfd_code *code, int n_frames, const float *v2c_dev,
                            float *c2v_dev, void *cuda_stream);

/* VARIABLE TO CHECK and TENTATIVE DECISION: lambda_vc = lambda0_v + lambda_c'v (c' the other
 * check of v) normalised to lambda_vc(0) = 0 (to the maximum where lambda_vc(0) = -inf);
 * symbols_dev [F][N] (may be NULL) = argmax_x lambda0_v + lambda_c1v + lambda_c2v, ties to the
 * lowest x. */
int nbfd_logsp_var_update(const nbfd_code *code, int n_frames, const float *llr_dev,
                          const float *c2v_dev, float *v2c_dev, uint16_t *symbols_dev,
                          void *cuda_stream);

/* ---- diagnostics (no counterpart in the paper) ----------------------------------------------
 * nbfd_diag_wait_expiry -- run the expiry path of the bounded device-side waits on purpose: one
 * thread waits, with the kernels' bounded mbarrier wait and a budget of budget_cycles SM cycles
 * (0 .. the kernels' own budget of 4e9), for bulk-copy bytes that are never sent. Nothing is in
 * flight and nothing faults; the call returns NBFD_ETIMEDOUT (the status nbfd_decode returns when
 * one of its waits expires) and the CUDA context stays usable. Synchronises `cuda_stream`. */
int nbfd_diag_wait_expiry(long long budget_cycles, void *cuda_stream);

/*
 * nbfd_diag_fp32_rate -- measured FP32 FMA rate of the device (no tensor cores), the peak the FP32
 * forms of the variable node are compared against: sm_count * blocks_per_sm blocks of 256
 * threads, each thread running 8 independent chains of `iters` FMAs (packed = 0: scalar fma.f32;
 * packed = 1: fma.f32x2, two lanes per instruction). One warm-up launch, then one launch timed
 * with CUDA events on `cuda_stream`. *tflops = 2 * FMAs / time (1e12 flop/s); *ms (may be NULL)
 * = the timed launch. blocks_per_sm in [1, 8], iters in [1, 2^30]. Synchronises `cuda_stream`.
 */
int nbfd_diag_fp32_rate(int packed, int blocks_per_sm, long long iters, double *tflops, double *ms,
                        void *cuda_stream);

/*
 * nbfd_diag_preset_status -- the next nbfd_decode or nbfd_decode_noalloc of the calling thread
 * starts its device status word (where a kernel whose bounded wait expired writes
 * NBFD_ETIMEDOUT) at `value` instead of 0; one-shot. The kernels only ever write that word, so the
 * decode runs as usual and a nonzero value must come back as NBFD_ETIMEDOUT: it shows on the host,
 * with no device fault, that an entry point reads its status word back. 0 cancels a preset.
 */
int nbfd_diag_preset_status(int32_t value);

/* Message for the calling thread's last failed call ("" if none). */
const char *nbfd_last_error(void);
/* Static name of a status code. */
const char *nbfd_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* NBFD_H */
