/*
 * conv.h - C ABI of the GB300 streaming partitioned-convolution engine.
 *
 * The engine runs the hot path of H. Rosseel and T. van Waterschoot,
 * "Accelerated Interactive Auralization of Highly Reverberant Spaces using
 * Graphics Hardware" (arXiv 2509.04390) entirely on one GPU:
 *
 *   synthesis   l(t) = H_aur^T * m~(t)            (Sec. 3.1, Eqs. 1-2)
 *   feedback    c(t) = F_hat * l(t)               (Sec. 3.1, Eq. 3)
 *   both as uniformly-partitioned overlap-save convolution with a
 *   frequency-domain delay line, n_f = 2 n_x      (Sec. 4, Eq. 6)
 *   the prediction over block n is subtracted from microphone block n+1
 *                                                 (Sec. 5)
 *
 * Every call returns CONV_OK (0) or a negative CONV_E_* code; the message of
 * the last failure on the calling thread is in conv_last_error().  Handles are
 * not thread-safe; separate handles are independent.  All float data are
 * row-major float32.  Host pointers are only read or written during the call
 * (the engine copies what it keeps); device pointers must stay valid until the
 * work enqueued on the given stream has finished.
 *
 * Output block n is exactly samples [n*block, (n+1)*block) of the causal
 * linear convolution with zero initial state; the engine adds no latency.
 */
#ifndef GB300_CONV_H
#define GB300_CONV_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CONV_OK 0
#define CONV_E_INVAL (-1)    /* bad argument or size                              */
#define CONV_E_STATE (-2)    /* call not valid in the handle's current state      */
#define CONV_E_NOMEM (-3)    /* device or pinned-host memory does not fit         */
#define CONV_E_CUDA (-4)     /* a CUDA runtime call failed (message has details)  */
#define CONV_E_TIMEOUT (-5)  /* a bounded device-side wait gave up                */
#define CONV_E_UNSTABLE (-6) /* closed-loop guard tripped; loop state was reset   */

/* storage precision of the filter and delay-line spectra (conv_set_precision) */
#define CONV_FP32 0 /* complex float32                                             */
#define CONV_FP16 1 /* complex float16 with power-of-two scales per (output tile,
                       partition) and per delay-line slot; FP32 FFTs and MAC     */
#define CONV_BF16 2 /* complex bfloat16, same scaling, FP32 FFTs and MAC           */

typedef struct conv_engine conv_engine; /* opaque; owns all device state */

/* Plan and size figures of a handle (conv_get_info).  Byte counts are the
 * algorithmic bytes one block moves through the named kernel. */
typedef struct conv_info {
    long long block;          /* n_x                                              */
    long long n_in;           /* inputs (microphones)                             */
    long long n_out;          /* outputs (loudspeakers)                           */
    long long taps;           /* n_h of the synthesis filters                     */
    long long K;              /* synthesis partitions of `block` taps: ceil(taps / block),
                                 or far_block / block with a far block          */
    long long taps_fb;        /* feedback-path length, 0 if none                  */
    long long K_fb;           /* feedback partitions, 0 if none                   */
    long long precision;      /* CONV_FP32 / CONV_FP16 / CONV_BF16                */
    long long mac_bytes;      /* synthesis tail MAC (partitions 1..K-1): filter
                                 spectra + delay-line rows, each read once      */
    long long mac_fb_bytes;   /* feedback FDL MAC, 0 if none                      */
    long long mac_ctas;       /* CTAs of one synthesis MAC launch                 */
    long long mac_splits;     /* partition splits per output tile                 */
    long long mac_smem;       /* dynamic shared memory per MAC CTA, bytes         */
    long long device_bytes;   /* device memory held by the handle                 */
    long long kernels_per_block;    /* kernels conv_process_block launches        */
    long long kernels_per_afc_block; /* kernels afc_process_block launches        */
    long long mac_bin_tile;   /* bins per MAC tile                                */
    long long mac_stages;     /* MAC pipeline depth                               */
    long long mac_stage_bytes; /* bytes per MAC pipeline stage                    */
    long long mac_warps;      /* MAC consumer warps                               */
    long long mac_kernel;     /* CONV_KERNEL_TMA / _DIRECT1 / _DIRECT2            */
    long long afc_adaptive;   /* 1 if the canceller adapts (afc_set_adaptation)   */
    long long far_block;      /* far block of non-uniform partitioning, 0 if none */
    long long K_far;          /* partitions of the far part                       */
    long long mac_far_bytes;  /* far tail MAC (once per far block), 0 if none    */
    long long fft_size;       /* n_f: 2 * block, or 3 * block in the spectrum-reuse
                                 form (afc_set_spectrum_reuse)                   */
    long long l2_keep_bytes;  /* tail filter spectra kept in L2 between blocks
                                 (conv_set_l2_keep)                              */
} conv_info;

/* Per-session counters (conv_get_stats).  Latency is the wall time of a
 * blocking host-buffer call (conv_process_block, afc_process_block) from entry
 * to return; the deadline is the block period block / fs. */
#define CONV_STATS_BUCKETS 24
typedef struct conv_stats {
    long long blocks;          /* blocks processed (every call form, batches included) */
    long long timed_calls;     /* blocking host-buffer calls that returned CONV_OK  */
    long long deadline_misses; /* timed calls that took longer than the block period */
    double max_latency_us;     /* longest timed call                               */
    double sum_latency_us;     /* sum over the timed calls (mean = sum / timed_calls) */
    long long latency_hist[CONV_STATS_BUCKETS]; /* timed calls by latency: bucket 0 holds
                                  [0, 2) us, bucket i in 1..22 holds [2^i, 2^(i+1)) us,
                                  bucket 23 everything from 2^23 us on               */
    long long device_errors;   /* device-side waits that gave up (CONV_E_TIMEOUT)  */
    long long guard_trips;     /* closed-loop guard trips (CONV_E_UNSTABLE)        */
} conv_stats;

/* Create an engine for n_in inputs, n_out outputs and filters of `taps` taps
 * at block size `block` (n_x, Sec. 4).  fs (Hz) only sets the block period
 * used in statistics.  block must be a power of two in [16, 4096] (the block
 * range of Sec. 6); n_in, n_out in [1, 1024]; taps >= 1.  Allocates all device
 * state on the current CUDA device (fails with NULL and conv_last_error() set,
 * e.g. when the footprint does not fit in free device memory).
 * Storage precision defaults to CONV_FP32. */
conv_engine* conv_create(double fs, int block, int n_in, int n_out, long long taps);

/* Choose the storage precision of filter and delay-line spectra (one of
 * CONV_FP32, CONV_FP16, CONV_BF16).  FFTs and accumulation stay FP32.  Only
 * valid before conv_set_filters (CONV_E_STATE afterwards).  Beyond the paper,
 * which keeps every spectrum in FP32: reduced-precision storage halves the
 * bytes the FDL MAC streams (each stored value is scaled by a power of two per
 * output tile and partition, or per delay-line slot, so scaling is exact). */
int conv_set_precision(conv_engine* e, int mode);

/* Spectrum-reuse form of the closed loop (the remark closing Sec. 5): on = 1
 * switches both convolutions to the FFT size n_f = 3 n_x, so that the
 * synthesis output spectrum, which then holds the last two output blocks
 * without wrap-around, enters the canceller's delay line as it is, and the
 * canceller's C_out input R2C transforms are saved.  Every spectrum of both
 * convolutions then has 3 n_x / 2 packed bins (1.5x the bytes each FDL MAC
 * streams).  The results equal those of the n_f = 2 n_x form up to rounding;
 * conv_process_block works too (a plain convolution at n_f = 3 n_x).
 * on = 0 returns to n_f = 2 n_x (the default).  Valid before conv_set_filters
 * and afc_set_paths (CONV_E_STATE afterwards); CONV_E_INVAL for block < 32;
 * CONV_E_STATE with a far block (conv_set_far_block), an adaptive canceller
 * (afc_set_adaptation with mu > 0) or while the session is in a batch, none
 * of which is combined with this form.  Re-allocates the synthesis spectra
 * and resets the engine's state. */
int afc_set_spectrum_reuse(conv_engine* e, int on);

/* FDL MAC kernels (conv_tiling.kernel) */
#define CONV_KERNEL_AUTO 0    /* planner's choice                                        */
#define CONV_KERNEL_TMA 1     /* producer warp streams 1-D bulk copies (TMA) into a ring */
#define CONV_KERNEL_DIRECT1 2 /* direct 16-byte loads, 1 partition in flight, 3 CTAs/SM (FP32 only;
                                 reduced precision falls back to CONV_KERNEL_TMA) */
#define CONV_KERNEL_DIRECT2 3 /* direct 16-byte loads, 2 partitions in flight, 2 CTAs/SM (FP32 only) */

/* Tiling of the synthesis FDL MAC; every field 0 = the planner's choice.
 *   kernel     CONV_KERNEL_*
 *   bin_tile   bins per tile, a power of two in [16, 256] (capped at block)
 *   stages     TMA ring depth, [2, 8]
 *   stage_kib  target bytes of filter spectra per TMA stage, KiB, [1, 96]
 *   splits     partition splits per tile (capped at what the tile allows)
 *   warps      TMA consumer warps, 8 or 16
 *   order      CONV_ORDER_*: how the TMA kernel's stages are dealt to splits */
typedef struct conv_tiling {
    int kernel, bin_tile, stages, stage_kib, splits, warps, order;
} conv_tiling;

#define CONV_ORDER_AUTO 0        /* planner's choice                                  */
#define CONV_ORDER_CONTIGUOUS 1  /* split s streams one contiguous range of stages    */
#define CONV_ORDER_INTERLEAVED 2 /* split s streams stages s, s+S, s+2S, ...          */

/* Fix the synthesis FDL MAC tiling instead of the planner's choice (the hook
 * the autotuner uses).  t may be NULL (all automatic).  Re-plans and
 * re-allocates; only valid before conv_set_filters and afc_set_paths
 * (CONV_E_STATE afterwards).  On failure the previous tiling is kept. */
int conv_set_tiling(conv_engine* e, const conv_tiling* t);

/* Set the synthesis filters H_aur (Sec. 3.1, Eq. 2): host array
 * h[n_out][n_in][taps] float32 (h[l][q] filters input q into output l).  The
 * engine partitions every filter into K sub-filters of `block` taps, pads each
 * with `block` zeros and takes its 2*block-point R2C FFT on the device (Sec. 4,
 * initialisation).  Copied; the caller keeps ownership.  Resets the stream. */
int conv_set_filters(conv_engine* e, const float* h);

/* Non-uniform partitioning (an extension: the paper, Sec. 3.2, considers
 * uniform partitions only).  far_block F (a power of two in (block, 4096])
 * splits every filter: taps [0, F) stay in this engine's partitions of
 * `block`; taps [F, taps) go to a second partitioned convolution of block F
 * that runs once every F / block blocks on the last F input samples.  Its
 * output over those samples, delayed by F, is added to the next F / block
 * output blocks.  The result is the same causal convolution (no added
 * latency).  The filter spectra streamed per output block drop from all
 * partitions to F + (taps - F) * block / F taps' worth.  0 turns it off.
 * Must come before conv_set_filters / afc_set_paths (CONV_E_STATE).  taps
 * must exceed F (CONV_E_INVAL).  Not combined with afc_set_adaptation,
 * afc_set_spectrum_reuse or batches (CONV_E_STATE).  With the feedback canceller, the far part filters
 * the error signal e, like the near part. */
int conv_set_far_block(conv_engine* e, int far_block);

/* The far part's engine of a non-uniformly partitioned engine (NULL if none).
 * Owned by `e`; use it only with conv_get_info, conv_profile_enable /
 * conv_profile_read (timing of the far tail MAC), and conv_set_far_block
 * before conv_set_filters on `e`: the far part then splits again (a third
 * partition size F2 > F for taps [F + F2, taps)), with the same result. */
conv_engine* conv_far_engine(conv_engine* e);

/* Set the a-priori feedback-path estimates F_hat (Sec. 3.1, Eq. 3): host array
 * f[n_in][n_out][taps_fb] float32 (f[p][l] is loudspeaker l -> microphone p).
 * Allocates the canceller's spectra and delay line.  Copied.  Resets the
 * stream. */
int afc_set_paths(conv_engine* e, const float* f, long long taps_fb);

/* Process one block, host buffers: in[n_in][block] -> out[n_out][block].
 * The three stages of Sec. 4: (1) slide the 2*block-sample input window by one
 * block and take its R2C FFT; (2) push the spectrum into the frequency-domain
 * delay line and multiply-accumulate every sub-filter spectrum with its
 * delay-line entry over all input -> output pairs (Eq. 6); (3) C2R IFFT and
 * keep the last `block` samples (overlap-save).
 * The block goes through the engine's mapped pinned host buffers, which the
 * pack kernel reads and the output kernel writes directly (no copy launches);
 * returns when out is written.  The next block's tail MAC keeps running in
 * the background.  Needs conv_set_filters (CONV_E_STATE otherwise). */
int conv_process_block(conv_engine* e, const float* in, float* out);

/* How the blocking host calls conv_process_block and afc_process_block
 * enqueue their work.  The graph form is one CUDA graph launch per call,
 * captured from the same kernels and launch shapes as the stream form on
 * first use.  conv_process_block's graph: pack -> output, and the next
 * block's tail MAC beside the output.  afc_process_block's (the static
 * canceller): pack -> output + push into the canceller's ring, the next
 * block's synthesis tail beside them, then the prediction for the next block
 * and the canceller's next tail.  The kernels read the block number from
 * device memory, which the graph's last node advances, so the arguments stay
 * the same from block to block.  The call returns when the graph's output is
 * on the host.  The stream form is the launches and their events, and starts
 * the pack while the previous block's tails may still run (the next launch
 * of a graph waits for the previous one, tails included).  Both forms give
 * the same bits.
 *   mode 1 (default): the graph when at least half a block period has
 *          passed since the previous call started (real-time use, one call
 *          per block period: the previous tails have finished), else the
 *          stream form (back-to-back calls);
 *   mode 2: the graph for every call;
 *   mode 0: the stream form for every call (drops the graphs).
 * A graph is rebuilt when the launch shapes change (a new plan).  Engines
 * with a far block, an adaptive canceller, the n_f = 3 n_x form, kernel
 * timing (conv_profile_enable) or batch membership always take the stream
 * form.  CONV_E_INVAL for another mode.  conv_get_host_graph reports the mode
 * and how many blocks went through a graph (never reset). */
int conv_set_host_graph(conv_engine* e, int mode);
int conv_get_host_graph(const conv_engine* e, int* mode, long long* graph_blocks);

/* n_blocks consecutive blocks from host buffers in one call (offline
 * rendering): in[n_in][n_blocks * block] and out[n_out][n_blocks * block],
 * row-major with row pitch n_blocks * block, owned by the caller.  The same
 * result as n_blocks calls of conv_process_block; the blocks run back to back
 * on the device in chunks of up to 256 blocks, with one strided copy in and
 * out per chunk (the chunk buffers are allocated on first use and kept).
 * Blocks until `out` is filled. */
int conv_process_blocks(conv_engine* e, const float* in, float* out, long long n_blocks);

/* Same as conv_process_block (the three stages of Sec. 4) with device
 * pointers d_in[n_in][block] and d_out[n_out][block], enqueued on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  Returns
 * once the work is enqueued.  Blocks of one engine form a chain: a block
 * enqueued on another stream than the previous block (or after a host-buffer
 * call) first waits for that stream's work.  d_out is complete in the order
 * of `cuda_stream`; the tail MAC of the next block, which the call also
 * enqueues, runs on the engine's background streams (conv_join_async). */
int conv_process_block_async(conv_engine* e, const float* d_in, float* d_out, void* cuda_stream);

/* Make `cuda_stream` wait for all work the engine has enqueued so far,
 * including the background tail MAC of the next block (and the canceller's,
 * the NLMS step's and the far engine's work), without blocking the host.
 * Work enqueued on `cuda_stream` afterwards starts once all of it is done:
 * for timing a run of blocks with CUDA events, or before reusing buffers the
 * engine may still read.  CONV_OK or CONV_E_INVAL / CONV_E_CUDA. */
int conv_join_async(conv_engine* e, void* cuda_stream);

/* One block of synthesis with feedback cancellation, host buffers:
 * e = mic - c_prev; out = H_aur^T * e; c = F_hat * out is kept and subtracted
 * from the next block (Sec. 5; the loop of Sec. 3.1, Fig. 1 and Eqs. 1-3, with
 * both convolutions run by the three stages of Sec. 4).  mic[n_in][block], out[n_out][block];
 * e_or_null (if not NULL) receives e[n_in][block].  Needs conv_set_filters and
 * afc_set_paths (CONV_E_STATE otherwise).  Returns CONV_E_UNSTABLE and resets
 * the loop state if the RMS of e exceeds the guard set by afc_set_guard. */
int afc_process_block(conv_engine* e, const float* mic, float* out, float* e_or_null);

/* Device-pointer form of afc_process_block, enqueued on `cuda_stream`.
 * d_e may be NULL.  The divergence guard is not evaluated (no host sync). */
int afc_process_block_async(conv_engine* e, const float* d_mic, float* d_out, float* d_e, void* cuda_stream);

/* Divergence guard of afc_process_block: if rms(e) over a block exceeds
 * `max_rms` (> 0), the call returns CONV_E_UNSTABLE and resets the loop
 * state.  0 disables the guard (the default). */
int afc_set_guard(conv_engine* e, double max_rms);

/* Adaptive feedback canceller.  An extension beyond the paper, whose F_hat
 * (Sec. 3.1, Sec. 5) is known in advance and static.  mu > 0 turns on a
 * partitioned-block frequency-domain NLMS update of the canceller's
 * sub-filter spectra; mu = 0 turns it off again (F_hat keeps its adapted value).
 *
 * Once per afc block n, after e_n = mic_n - c_{n-1} is formed and before l_n
 * enters the canceller's delay line:
 *   E_p    = R2C_2B([0_B | e_n,p])               (B zeros, then the error block)
 *   pow[k] = lambda pow[k] + (1 - lambda) sum_l |U_l,0[k]|^2
 *   F_hat[p][l][j][k] += mu E_p[k] conj(U_l,j[k]) / (K_fb pow[k] + delta)
 * U_l,j: R2C of loudspeaker l's 2B-sample window of block n-1-j (the delay
 * line that produced c_{n-1}).  The update is unconstrained: it does not
 * project F_hat back onto B-tap sub-filters.  The packed bin 0 holds DC and
 * Nyquist, and each is updated with its own power.  pow starts at 0, and
 * conv_reset sets it back to 0.  conv_reset keeps the adapted F_hat.
 * afc_set_paths restores a given estimate.  c_n is computed with the
 * updated F_hat.  (Internally, partition 0 takes each step at once and the
 * other partitions two blocks later, with correction terms that give the same
 * c_n; afc_get_path_spectra and turning adaptation off first apply what is
 * pending.)
 *
 * mu in [0, 2), lambda in [0, 1), delta >= 0 finite (> 0 when mu > 0), else
 * CONV_E_INVAL.  CONV_E_STATE without afc_set_paths, for FP16/BF16 engines
 * (the update needs FP32 spectra), in the spectrum-reuse form (mu > 0), or
 * while the session is in a batch.
 * Waits for the engine's queued work.  Takes effect from the next block.
 * While adaptation is on, the conv_process_* calls (synthesis only) return
 * CONV_E_STATE: every block must pass through the canceller. */
int afc_set_adaptation(conv_engine* e, double mu, double lambda, double delta);

/* Copy the canceller's current sub-filter spectra to host memory f_spec, laid
 * out [n_in (mic p)][n_out (loudspeaker l)][K_fb][block] complex values as
 * (re, im) float pairs: 2 * n_in * n_out * K_fb * block floats, owned by the
 * caller.  Bin 0 holds (DC, Nyquist).  The values are 2B-point R2C
 * spectra of the zero-padded sub-filters, unscaled (Sec. 4 initialisation).
 * Waits for the engine's queued work.  CONV_E_STATE without afc_set_paths,
 * for FP16/BF16 engines, or in the spectrum-reuse form. */
int afc_get_path_spectra(conv_engine* e, float* f_spec);

/* Zero the delay lines, sliding windows and the pending feedback prediction
 * (start of a new stream): the zero initial state that the causal convolution
 * of Sec. 3.1 (Eq. 2) and the loop of Sec. 5 start from.  Filters and feedback
 * paths are kept (an adapted F_hat too).  Waits for the engine's queued work.
 * Also the way back after CONV_E_TIMEOUT or CONV_E_UNSTABLE. */
int conv_reset(conv_engine* e);

/* Wait for all work the engine enqueued and report a device-side error
 * (CONV_E_TIMEOUT if a bounded wait gave up). */
int conv_synchronize(conv_engine* e);

/* Copy the handle's counters (conv_stats) to *out; conv_reset_stats zeroes
 * them.  The counters survive conv_reset. */
int conv_get_stats(const conv_engine* e, conv_stats* out);
int conv_reset_stats(conv_engine* e);

/* Fault-path testing of the bounded device-side waits.  The next synthesis
 * tail MAC this handle launches has one CTA's producer withhold its first
 * pipeline stage (it issues no copy and no arrival for it), so that CTA's
 * consumers wait on a barrier that nothing completes.  Their wait is bounded
 * by wait_ns (in [1e3, 1e9]) for that launch: they give up, raise the CTA's
 * abort flag, record the error and return; the producer lets its other copies
 * land first.  No GPU fault and no hang: the context stays usable.  The call
 * whose output uses that tail returns CONV_E_TIMEOUT (its results, and those
 * of blocks after it, are invalid until conv_reset).  CONV_E_STATE before
 * conv_set_filters, with one partition (no tail MAC) or with the direct-load
 * MAC (it has no pipeline waits). */
int conv_inject_wait_timeout(conv_engine* e, long long wait_ns);

/* Fill *out with the plan and size figures of the handle. */
int conv_get_info(const conv_engine* e, conv_info* out);

/* Kernel timing: while enabled, every block records CUDA events around the
 * synthesis FDL MAC kernel on the stream it is launched on, and consecutive
 * MAC launches are kept from overlapping (so each duration is the kernel's
 * own).  conv_profile_read
 * waits for the recorded work, returns the summed kernel time in milliseconds
 * and the number of launches timed, and clears the record. */
int conv_profile_enable(conv_engine* e, int enable);
int conv_profile_read(conv_engine* e, double* mac_ms_total, long long* launches);

/* L2 residency of the filter spectra between blocks: the tail MACs stream
 * the first `bytes` of their filter spectra (partitions 1.. in order; the
 * canceller's first, then the synthesis') with the L2 evict-last policy, so
 * that the next block reads them from L2, and the rest with evict-first.
 * Default 56 MB: at the paper configuration on GB300 (136 MB L2), 52-60 MB
 * gave the shortest back-to-back steps (FP32 27.4 -> 23.0 us, FP16 16.7 ->
 * 15.6 us) and more gave longer ones.  0 streams everything evict-first (for
 * example when several engines run at once).  Results do not depend on it.
 * Takes effect from the next block; CONV_E_INVAL for bytes < 0.  Batched
 * sessions always stream evict-first. */
int conv_set_l2_keep(conv_engine* e, long long bytes);

/* Profiling aid: while kernel timing is enabled, read `bytes` of a zeroed
 * scratch buffer (allocated here, owned by the handle) on the MAC's stream
 * before each timed MAC launch, outside its events, so that a working set
 * smaller than the L2 cache does not start the launch with its data still
 * cached (reading leaves clean lines: no write-back lands in the timed
 * launch).  Pass a few times the L2 size.  0 turns it off and frees the
 * buffer.  CONV_E_NOMEM if the buffer cannot be allocated. */
int conv_profile_flush_l2(conv_engine* e, long long bytes);

/* Host-only dry run of the kernel tiling the engine would choose for these
 * sizes: replays the FDL MAC kernel's copy and store addresses for every CTA
 * and stage against the buffer and shared-memory sizes.  Needs no device.
 * precision is CONV_FP32/FP16/BF16, n_src/n_dst the convolution's inputs and
 * outputs, num_sms the SM count to plan for, t the conv_set_tiling override
 * (NULL = planner).  CONV_OK or CONV_E_INVAL. */
int conv_plan_check(int precision, int block, int n_src, int n_dst, long long taps, int num_sms,
                    const conv_tiling* t);

/* FDL MAC and output transform of one block over caller-owned buffers,
 * allocating nothing.  (The paper has no counterpart: this serves callers that
 * cannot allocate device memory, such as a real-time audio callback, where an
 * allocation can block past the block deadline, or a plugin whose host owns
 * every device buffer.)
 *
 * Computes y[l][t] = the last `block` samples of the 2*block-point C2R IFFT
 * (scaled 1/(2*block)) of  sum_p sum_q H[p][q][l] * X[(slot0 + p) mod K][q],
 * i.e. stages 2 and 3 of the engine for one block, with the spectra given:
 *   d_H  device, [K][n_in][n_out][block] complex float (re, im interleaved):
 *        the 2*block-point R2C spectra of the zero-padded sub-filters, packed
 *        (bin 0 holds (DC, Nyquist) as (re, im); bins 1..block-1 as usual);
 *   d_X  device, [K][n_in][block] complex float, packed the same way: the
 *        delay-line ring; slot0 is the slot of the newest input spectrum and
 *        partition p reads slot (slot0 + p) mod K;
 *   d_y  device, [n_out][block] float, written.
 * d_H and d_X must be 16-byte aligned (the spectra are streamed with bulk
 * copies that need it), d_y 4-byte aligned; CONV_E_INVAL otherwise, before
 * anything is launched.
 * Enqueued on `cuda_stream` (NULL = legacy default stream); d_H and d_X must
 * be complete in stream order.  FP32 only.  Limits: block a power of two in
 * [16, 256], n_out in [1, 16], n_in*K <= 2^30; CONV_E_INVAL beyond them.
 *
 * The split partials live in a 2 MiB file-scope device array (plus 8 KB of
 * twiddle tables and an error word) that every GPU loading this library holds
 * until exit.  The first call on a device, with that device current, resolves
 * the arrays' device addresses and uploads the twiddles; make that first call
 * before any stream capture.  All calls share the array, and every call
 * writes all the partials it reads, so nothing needs clearing; calls that
 * overlap on the GPU race on the array.  Returns CONV_OK or a negative
 * CONV_E_* code with the message in conv_last_error().  The call returns once
 * the work is enqueued, so a bounded device-side wait that gives up is not
 * known yet: conv_fdl_mac_noalloc_status reports it. */
int conv_fdl_mac_noalloc(const float* d_H, const float* d_X, int block, int n_in, int n_out, long long K,
                         long long slot0, float* d_y, void* cuda_stream);

/* Error report of conv_fdl_mac_noalloc on the current device: waits for the
 * work enqueued on `cuda_stream`, then reads and clears the device's error
 * word.  CONV_E_TIMEOUT if a bounded wait of any call since the last report
 * gave up (that call's output is invalid), else CONV_OK.  Allocates nothing. */
int conv_fdl_mac_noalloc_status(void* cuda_stream);

/* Device bytes a handle with these sizes would hold (synthesis, plus the
 * feedback canceller when taps_fb > 0), from the same planner the engine
 * uses; host-only, allocates nothing.  For admission control.  -1 with
 * conv_last_error() on invalid sizes. */
long long conv_footprint(int precision, int block, int n_in, int n_out, long long taps, long long taps_fb,
                         int num_sms);

/* ---------------------------------------------------------------- batches
 * A batch processes one block of each of many independent sessions per step
 * with one launch per stage for all of them (batched pack + R2C, batched
 * head + output, batched tail MAC for the next block), whatever their block
 * sizes, channel counts, filter lengths and tilings.  Sessions keep their own
 * state; a session in a batch must not be processed on its own (add/remove
 * hand it over).  All sessions of a batch share the batch's precision and use
 * the TMA MAC with 8 consumer warps.  Sessions with feedback paths run the
 * canceller too (Sec. 5): their input is the microphone block. */
typedef struct conv_batch conv_batch;

/* Create an empty batch for sessions of the given precision on the current
 * device.  NULL on failure (conv_last_error()). */
conv_batch* conv_batch_create(int precision);

/* Add a session (filters set; feedback paths, if allocated, set too).  Waits
 * for the session's own outstanding work and the batch's.  Sessions with a far
 * block, an adaptive canceller or in the spectrum-reuse form are not batched
 * (CONV_E_STATE). */
int conv_batch_add(conv_batch* b, conv_engine* e);

/* Remove a session; it can be processed on its own again afterwards. */
int conv_batch_remove(conv_batch* b, conv_engine* e);

/* Number of sessions. */
int conv_batch_size(const conv_batch* b);

/* One block of every session, in the order they were added: d_in[i] is the
 * device buffer [n_in_i][block_i] of session i, d_out[i] its output
 * [n_out_i][block_i].  d_in/d_out are host arrays of device pointers, read
 * during the call.  Enqueued on `cuda_stream` (NULL: the batch's own
 * stream); returns once enqueued.  Consecutive calls must use the same
 * stream. */
int conv_batch_process_async(conv_batch* b, const float* const* d_in, float* const* d_out, void* cuda_stream);

/* One block of `count` of the sessions: idx[j] is the index (in add order) of
 * the j-th session to process, d_in[j] / d_out[j] its buffers.  The others
 * keep their state and can be processed in a later call (sessions with
 * different block periods come due on different steps).  Same stream rules
 * as conv_batch_process_async. */
int conv_batch_process_some_async(conv_batch* b, int count, const int* idx, const float* const* d_in,
                                  float* const* d_out, void* cuda_stream);

/* Persistent batch steps.  mode 1: every later step of the batch runs as ONE
 * kernel launch instead of one launch per stage; mode 2: the same, replayed
 * from a CUDA graph (the step's table copy, counter reset and launch, captured
 * once per table layout and replayed while the due sessions and table sizes
 * stay the same: the graph's copy reads the step's freshly built table);
 * mode 0: back to one launch per stage.  About one CTA per SM claims
 * work items from a device-side list in dependency order: the synthesis
 * packs, then the outputs, the canceller's packs and outputs, then the tail
 * MACs of the next block.  An item that needs other items' results waits for
 * a device counter they raise.  Every such wait is bounded; a wait that gives
 * up is reported as CONV_E_TIMEOUT by conv_batch_synchronize.  The items run
 * the same device code as the separate launches, so the outputs are the same
 * bit for bit.  The step's argument tables and work list are built on the
 * host and copied in with one copy, as in the other mode.  Can be switched
 * between steps.  CONV_OK or CONV_E_INVAL / CONV_E_CUDA. */
int conv_batch_set_persistent(conv_batch* b, int mode);

/* Wait for all of the batch's work; report a device-side error of any session. */
int conv_batch_synchronize(conv_batch* b);

/* Make `cuda_stream` wait for all the batch's work so far, including the
 * background tail MACs of the next step (no host wait). */
int conv_batch_join_async(conv_batch* b, void* cuda_stream);

/* Algorithmic bytes of one step's batched tail MAC (all sessions, both
 * convolutions of canceller sessions). */
long long conv_batch_step_bytes(const conv_batch* b);

/* Free the batch (its sessions are left intact and usable on their own).  NULL-safe. */
void conv_batch_destroy(conv_batch* b);

/* ------------------------------------------------------ shared-filter groups
 * A group runs `sessions` streams that use one filter set (same block, n_in,
 * n_out, taps) in lock-step: one call processes block n of every session.
 * For every bin k the FDL MAC of Sec. 4 (Eq. 6) over all sessions is then one
 * complex GEMM, Y_k[l][s] = sum over (p, q) of H_k[l][q][p] X_k,s[q][(head - p) mod K],
 * which runs on the tensor cores (FP16 or BF16 operands, FP32 accumulation)
 * and reads every filter spectrum once per block for all sessions.  This is
 * an extension beyond the paper, which runs one stream per engine.
 *
 * Limits (else CONV_E_INVAL): precision CONV_FP16 or CONV_BF16; n_out in
 * {8, 16, 32}; n_in in {1, 2, 4, 8}; sessions 1, 2, 4 or a multiple of 8,
 * with sessions * 128 / n_out in [8, 128]; block a power of two in
 * [16, 4096].  A group of one session is a single stream whose MAC runs on
 * the tensor cores.
 * Filter spectra carry a power-of-two scale per (bin, output); the delay line
 * is stored unscaled, so FP16 groups saturate input spectra above 65504
 * (inputs with |x| <= 1 never reach it: |X| <= 2 * block).  Output block n of
 * every session is exactly samples [nB, (n+1)B) of its causal convolution,
 * as for conv_process_block.  The schedule is the engine's split phase: the
 * tail MAC (all K-steps but the first) of block n+1 runs on background
 * streams as soon as block n's spectra are in the delay lines, and a block's
 * call runs the pack, then the first K-step (on CUDA cores) with the tail's
 * partials and the C2R output; far higher throughput per GPU than separate
 * engines. */
typedef struct conv_group conv_group;

typedef struct conv_group_info {
    long long block, n_in, n_out, taps, sessions, precision;
    long long K;              /* partitions                                       */
    long long ring_slots;     /* delay-line slots (K rounded up to a K-step)      */
    long long bins_per_group; /* bins per tensor-core tile (128 / n_out)          */
    long long groups;         /* bin groups (block / bins_per_group)              */
    long long splits;         /* partial slots per bin group (most MAC CTAs sharing one group) */
    long long k_steps;        /* K-steps of 16 reduction indices per block        */
    long long stage_k_steps;  /* K-steps per pipeline stage                       */
    long long stages;         /* pipeline depth                                   */
    long long mac_ctas;       /* CTAs of one MAC launch                           */
    long long mac_smem;       /* dynamic shared memory per MAC CTA, bytes         */
    long long tmem_cols;      /* tensor-memory columns per MAC CTA                */
    long long mac_bytes;      /* algorithmic bytes of one MAC launch: filters + delay lines, each read once */
    long long device_bytes;   /* device memory held                               */
    long long kernels_per_block; /* kernels one process call launches             */
    long long tail_streams;   /* background streams of the tails                  */
    long long tail_ctas;      /* CTAs of one MAC launch (= mac_ctas)              */
    long long acc_buffers;    /* TMEM accumulator buffers per MAC CTA             */
} conv_group_info;

/* Tiling of a group's tensor-core MAC (autotuner hook); 0 leaves a field to
 * the planner.  ctas: MAC CTAs, at most one per SM (default: one per SM),
 * each taking an equal run of (bin group, K-step) units; stage_k_steps: 1..4;
 * stages: 2..8; tail_streams: 1 (tails of consecutive blocks in order on one
 * stream) or 2 (alternating streams, consecutive tails may overlap). */
typedef struct conv_group_tiling {
    int ctas, stage_k_steps, stages, tail_streams;
} conv_group_tiling;

/* Create a group on the current device; NULL on failure (conv_last_error()). */
conv_group* conv_group_create(int precision, int block, int n_in, int n_out, long long taps, int sessions);

/* Same with a tiling (NULL: the planner's choice). */
conv_group* conv_group_create_tiled(int precision, int block, int n_in, int n_out, long long taps, int sessions,
                                    const conv_group_tiling* tiling);

/* Host filters h[n_out][n_in][taps] (copied; caller keeps ownership), shared
 * by all sessions.  Resets the sessions' state. */
int conv_group_set_filters(conv_group* g, const float* h);

/* One block of every session: d_in [sessions][n_in][block] and
 * d_out [sessions][n_out][block], device pointers, enqueued on `cuda_stream`
 * (NULL: the legacy default stream).  CONV_E_STATE before conv_group_set_filters. */
int conv_group_process_async(conv_group* g, const float* d_in, float* d_out, void* cuda_stream);

/* Same with host buffers; blocks until the outputs are in `out`.  Reports a
 * device-side wait that gave up as CONV_E_TIMEOUT. */
int conv_group_process(conv_group* g, const float* in, float* out);

/* n_blocks consecutive blocks of every session from host buffers in one call:
 * in [sessions][n_in][n_blocks * block], out [sessions][n_out][n_blocks * block]
 * (row pitch n_blocks * block), owned by the caller.  The same result as
 * n_blocks calls of conv_group_process; chunks of up to 256 blocks run back to
 * back on the device, one strided copy in and out per chunk. */
int conv_group_process_blocks(conv_group* g, const float* in, float* out, long long n_blocks);

/* Zero every session's delay line and window (filters kept). */
int conv_group_reset(conv_group* g);

/* Wait for the group's work; CONV_E_TIMEOUT if a device-side wait gave up. */
int conv_group_synchronize(conv_group* g);

/* Make `cuda_stream` wait for all the group's work so far, including the
 * background tail MAC of the next block (no host wait). */
int conv_group_join_async(conv_group* g, void* cuda_stream);

int conv_group_get_info(const conv_group* g, conv_group_info* out);

/* Host-only: plans a group and replays every copy address of a block against
 * the buffer and shared-memory sizes.  CONV_OK or CONV_E_INVAL with the reason. */
int conv_group_plan_check(int precision, int block, int n_in, int n_out, long long taps, int sessions, int num_sms,
                          const conv_group_tiling* tiling);

/* CUDA-event timing of each MAC launch (enable > 1: number of event pairs),
 * read and cleared by conv_group_profile_read (total ms, launches). */
int conv_group_profile_enable(conv_group* g, int enable);

/* L2 residency of the group's filter tiles between blocks (as conv_set_l2_keep
 * for one engine): the first `bytes` of them (the lowest partitions of every
 * bin group) are streamed with the L2 evict-last policy, the rest and the
 * delay lines evict-first.  Default 60 MB (measured at 8 sessions of the paper
 * configuration, FP16: 29.3 -> 26.5 us per step).  0 turns it off; results do
 * not depend on it.  CONV_E_INVAL for bytes < 0. */
int conv_group_set_l2_keep(conv_group* g, long long bytes);
int conv_group_profile_read(conv_group* g, double* total_ms, long long* launches);

/* Free everything the group owns.  NULL-safe. */
void conv_group_destroy(conv_group* g);

/* Free everything the handle owns.  NULL-safe. */
void conv_destroy(conv_engine* e);

/* Message of the last failure on the calling thread ("" if none). */
const char* conv_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300_CONV_H */
