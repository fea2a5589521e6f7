/*
 * pvf.h -- C ABI of the GB300 (sm_103a) PVFinder inference library (libpvf.so).
 *
 * The library runs the inference hot path of the hybrid PVFinder algorithm of
 * arXiv 2602.19959 on one GPU, every step in hand-written CUDA kernels:
 *   1. per-track fully connected network on nine track features        (§2)
 *   2. deterministic scatter-sum of the track outputs into each event's
 *      4000-bin z histogram (40 slices x 100 bins over [-100, 300) mm)   (§2)
 *   3. UNet-style 1D CNN over the histogram                              (§2)
 *   4. peak finding (local maximum + threshold + centroid)               (§2)
 * It follows the deployment constraints of §3: zero-copy Structure-of-Arrays
 * input, one fixed caller-owned device pool bound at creation (nothing is
 * allocated afterwards), execution on the caller's single stream with no
 * default-stream work and no device-wide synchronisation inside pvf_infer, and
 * deterministic results (no floating-point atomics; every per-bin sum has a fixed
 * order that depends only on the event's own tracks).
 *
 * Conventions for every function below:
 *   - Pointers documented as "device" must point to device memory (or memory the
 *     device can access); "host" pointers are read on the calling thread.
 *   - Functions return PVF_OK or an error code and never abort the process.
 *     Argument errors are detected on the host before any work is enqueued, and
 *     nothing is enqueued when a function returns an error.
 *   - Work is enqueued on the given stream and the call returns after enqueueing,
 *     unless the function says it synchronises.
 *   - A handle may be used from one thread at a time. Calls that overlap on the
 *     device (different streams, same handle) race on the handle's pool.
 */
#ifndef PVF_H
#define PVF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PVF_API __attribute__((visibility("default")))
#else
#define PVF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without including the CUDA headers. */
typedef struct CUstream_st *pvf_stream_t;

/* Status codes (§3: "Error handling employs a Status enum enabling graceful
 * degradation"). Values >= PVF_WARN_EVENTS_SKIPPED are warnings: results were
 * produced, but some events were bypassed or truncated. */
typedef enum {
    PVF_OK = 0,
    PVF_ERR_INVALID_ARG = 1,     /* null/misaligned pointer, size out of range        */
    PVF_ERR_POOL_TOO_SMALL = 2,  /* pool smaller than pvf_pool_bytes_required         */
    PVF_ERR_WEIGHTS = 3,         /* weight blob malformed or of another architecture  */
    PVF_ERR_CUDA = 4,            /* a CUDA runtime call failed                        */
    PVF_ERR_TIMEOUT = 5,         /* a bounded device-side wait gave up                */
    PVF_ERR_UNSUPPORTED = 6,     /* feature not available for this configuration      */
    PVF_WARN_EVENTS_SKIPPED = 16,/* some events were bypassed (count = -1)            */
    PVF_WARN_TRUNCATED = 17      /* some event had more than max_pv_per_event PVs     */
} pvf_status;

/* Arithmetic of the FC net and of the UNet convolutions. The histogram, the first
 * (1 -> c0 channel) convolution, the final convolution, the sigmoid and the
 * centroids are float32 in every form. */
typedef enum {
    PVF_FP32 = 0,      /* CUDA-core float32 ("plain FP32 GPU form")                     */
    PVF_BF16 = 1,      /* tcgen05 tensor cores, bf16 operands, fp32 accumulation         */
    PVF_FP8_E4M3 = 2,  /* tcgen05 tensor cores, e4m3 operands with per-output-channel
                          weight scales and per-tensor activation scales, fp32 accum.   */
    PVF_FP16 = 3       /* tcgen05 tensor cores, f16 operands, fp32 accumulation: the
                          mixed-precision form proposed in §5 (Table 2). Stored values beyond
                          the f16 range saturate to +-65504 (NaN stays NaN).           */
} pvf_precision;

/* Launch schedule: how many CTAs per SM each persistent kernel family launches (its grid
 * is that times the SM count, capped by its work). 0 = as many as fit at once (the
 * default); values above what fits are clamped to it. These are the autotuner's
 * parameters (the events per CTA of the front follow from its grid); results do not
 * depend on them. */
typedef struct {
    int32_t front_ctas_per_sm;     /* front kernel (steps 1-2 + enc1), tensor-core forms:
                                      1-2 run 256-thread CTAs (FC passes of 256 tracks), 3-4
                                      128-thread CTAs (passes of 128 tracks); 0 = 2 for
                                      launches of at most 4 events per SM, else 4. The
                                      float32 front: 1..2                                   */
    int32_t conv_ctas_per_sm[6];   /* tensor-core forms: enc2, enc3, enc4_up3, dec3_up2,
                                      dec2_up1, dec1_final                                    */
    int32_t tail_ctas_per_sm;      /* peak finder: 1..8                                         */
} pvf_schedule;

/* Creation-time plan (§3: TensorSpec freezing batch dimensions, channels, length and
 * data type at initialisation). Everything is frozen at pvf_create. */
typedef struct {
    int32_t precision;             /* pvf_precision                                        */
    int32_t max_events;            /* largest n_events of one pvf_infer call, >= 1          */
    int32_t max_tracks_per_event;  /* 1..8192; larger events are bypassed (count = -1)      */
    int32_t max_pv_per_event;      /* output slots per event, 1..1024                       */
    int32_t chunk_events;          /* events whose UNet activations are resident at once;
                                      0 = max_events. Smaller chunks shrink the pool.       */
    float boundary_mm;             /* §3 boundary tracks: 0 = every track fills its own
                                      slice only. 0 < w < 5: a track whose slice-relative
                                      z (float32, z - (-100 + 10 s)) is < w also fills slice
                                      s - 1, one >= 10 - w (float32) also slice s + 1, with
                                      feature 2 relative to the slice it fills; none below
                                      slice 0 or above 39. Other values: INVALID_ARG.      */
    int32_t unet_width;            /* UNet base width c0 (levels c0, 2c0, 4c0, 8c0): 0 or 16
                                      = the 16/32/64/128 network; 32 = the wide 32/64/128/256
                                      variant (§5's channel-count axis), every form. Must
                                      match the blob's width (else pvf_create returns
                                      ERR_WEIGHTS). Other values: INVALID_ARG.              */
    int32_t per_interval;          /* 0: the UNet runs over each event's 4000 bins. 1: the
                                      §3 per-interval layout -- each of the 40 intervals runs
                                      as its own 104-bin sequence (its 100 bins and two zero
                                      bins on each side) and its 100 central logits fill the
                                      interval's bins. Every form, width 16 only (width 32:
                                      UNSUPPORTED). Other values: INVALID_ARG.              */
    const float *fp8_act_scales;   /* host, PVF_FP8_E4M3 only: PVF_N_ACT_SCALES per-tensor
                                      input scales (amax / 448), or NULL to use
                                      pvf_calibrate before the first pvf_infer              */
    const pvf_schedule *schedule;  /* host, copied at pvf_create, or NULL: the defaults (a
                                      table written by the autotuner goes here); negative
                                      entries: INVALID_ARG                                   */
} pvf_config;

#define PVF_N_FEATURES 9
#define PVF_N_BINS 4000
#define PVF_N_ACT_SCALES 16

/* Track features, Structure of Arrays (§3: Allen's SoA buffers, read zero-copy).
 * f[k] points to a device float array of n_tracks entries indexed by global track
 * number, in the order poca_x, poca_y, poca_z, tx, ty, w1, w2, w3, quality. Events
 * whose offsets reach past n_tracks are bypassed, never read. */
typedef struct {
    const float *f[PVF_N_FEATURES];
    int64_t n_tracks;
} pvf_tracks_soa;

typedef struct pvf_handle pvf_handle;

/* Bytes of device pool that pvf_create needs for cfg (weights, per-event state and
 * activations, with 256-byte alignment slack). Host only; no CUDA call. */
PVF_API pvf_status pvf_pool_bytes_required(const pvf_config *cfg, size_t *out_bytes);

/* Creates a handle.
 *   weights_blob  host, blob_bytes bytes: float32 master weights in the "PVFW" v1
 *                 format (header, layer table, data); copied, caller keeps ownership.
 *   pool          device, >= pvf_pool_bytes_required(cfg) bytes, 256-byte aligned;
 *                 caller-owned, never freed by the library, must outlive the handle.
 *   stream        stream used for the one-time upload; pvf_create synchronises it.
 * The weights are converted to the chosen precision and laid out in the pool;
 * no device memory is allocated by the library, now or later.
 * Errors: PVF_ERR_INVALID_ARG, PVF_ERR_WEIGHTS, PVF_ERR_POOL_TOO_SMALL, PVF_ERR_CUDA. */
PVF_API pvf_status pvf_create(const void *weights_blob, size_t blob_bytes, void *pool,
                      size_t pool_bytes, const pvf_config *cfg, pvf_stream_t stream,
                      pvf_handle **out);

/* Runs the whole path on n_events events (0 <= n_events <= max_events).
 *   tracks        features of all tracks (device arrays, see pvf_tracks_soa)
 *   event_offsets device int32[n_events + 1]; event e owns tracks
 *                 [event_offsets[e], event_offsets[e+1])
 *   out_pv_z      device float[n_events * max_pv_per_event]: PV z in mm, ascending
 *                 per event; slots past the event's count are left untouched
 *   out_pv_count  device int32[n_events]: number of PVs found (may exceed
 *                 max_pv_per_event: only the first max_pv_per_event z are written),
 *                 or -1 when the event was bypassed
 * An event is bypassed (§3: events failing validation bypass ML reconstruction)
 * when its offsets are negative, decreasing or beyond tracks->n_tracks, or it has
 * more than max_tracks_per_event tracks. A track is dropped (not an error) when a feature is
 * not finite or its z lies outside [-100, 300) mm. Warnings are reported by
 * pvf_last_device_status. Asynchronous on stream. */
PVF_API pvf_status pvf_infer(pvf_handle *h, const pvf_tracks_soa *tracks,
                     const int32_t *event_offsets, int32_t n_events, float *out_pv_z,
                     int32_t *out_pv_count, pvf_stream_t stream);

/* pvf_infer that also copies intermediate results, for parity checks:
 *   out_hist   device float[n_events * 4000] or NULL: the histogram (step 2)
 *   out_logit  device float[n_events * 4000] or NULL: the final conv output before
 *              the sigmoid (step 3); peak decisions are taken on these logits */
PVF_API pvf_status pvf_infer_ex(pvf_handle *h, const pvf_tracks_soa *tracks,
                        const int32_t *event_offsets, int32_t n_events, float *out_pv_z,
                        int32_t *out_pv_count, float *out_hist, float *out_logit,
                        pvf_stream_t stream);

/* Stage entry points: the same kernels as pvf_infer, one step at a time.
 * pvf_stage_histogram: steps 1-2 -> out_hist device float[n_events * 4000].
 * pvf_stage_unet:      step 3 on a given histogram (device float[n_events * 4000])
 *                      -> out_logit device float[n_events * 4000] (pre-sigmoid).
 * pvf_stage_peaks:     step 4 on given logits (device float[n_events * 4000]). */
PVF_API pvf_status pvf_stage_histogram(pvf_handle *h, const pvf_tracks_soa *tracks,
                               const int32_t *event_offsets, int32_t n_events,
                               float *out_hist, pvf_stream_t stream);
PVF_API pvf_status pvf_stage_unet(pvf_handle *h, const float *hist, int32_t n_events,
                          float *out_logit, pvf_stream_t stream);
PVF_API pvf_status pvf_stage_peaks(pvf_handle *h, const float *logit, int32_t n_events,
                           float *out_pv_z, int32_t *out_pv_count, pvf_stream_t stream);

/* FP8 calibration (the per-tensor activation scales of PVF_FP8_E4M3). Runs steps 1-3
 * of a PVF_BF16 handle on n_events calibration events while recording max |x| of every
 * activation tensor that the FP8 form stores, and writes out_scales[i] = amax_i / 448
 * (1 where amax_i = 0) for i < PVF_N_ACT_SCALES (unused slots = 1): the value to pass as
 * pvf_config.fp8_act_scales. Slots: 0 e1/p1/u1, 1 e2/p2/u2, 2 e3/p3/u3 (the halves of
 * each skip concat share a scale), 3 e4, 4 d3, 5 d2, 6 d1.
 *   out_scales  host float[PVF_N_ACT_SCALES]
 * Errors: PVF_ERR_UNSUPPORTED unless h is a PVF_BF16 handle. Synchronises stream. */
PVF_API pvf_status pvf_calibrate(pvf_handle *h, const pvf_tracks_soa *tracks,
                                 const int32_t *event_offsets, int32_t n_events,
                                 float *out_scales, pvf_stream_t stream);

/* Reads and clears the handle's device status word (the worst status raised by
 * kernels since the last read: PVF_OK, PVF_WARN_*, PVF_ERR_TIMEOUT).
 * Synchronises stream. */
PVF_API pvf_status pvf_last_device_status(pvf_handle *h, int32_t *out_status, pvf_stream_t stream);

/* Failure detection (§3 bounds every device-side wait; the paper has no test counterpart):
 * runs the tensor-core enc2 kernel on the handle's first n_events events with its MMA
 * thread waiting, for limit_us microseconds, on a barrier that nothing arrives on. The wait
 * gives up, the kernel raises PVF_ERR_TIMEOUT in the device status word, waits (bounded)
 * for its own copies in flight, frees its tensor memory and returns; the handle stays
 * usable. For tests of the bounded-wait path (every production wait gives up after 1 s).
 *   n_events  1..min(max_events, chunk_events); limit_us 1..100000
 * Errors: PVF_ERR_INVALID_ARG; PVF_ERR_UNSUPPORTED for PVF_FP32 (no tensor-core waits).
 * Asynchronous on stream; read the status with pvf_last_device_status. The kernel writes
 * the handle's activation buffers: run pvf_infer again before reading results. */
PVF_API pvf_status pvf_test_wait_timeout(pvf_handle *h, int32_t n_events, uint32_t limit_us,
                                         pvf_stream_t stream);

/* Per-kernel timing (CUDA events recorded around every kernel launch on the launch
 * stream), for profiling only. pvf_profile_enable(h, 1) creates the events (host-side
 * driver objects, no device memory) and starts recording; 0 stops. */
typedef struct {
    char name[24];       /* kernel family, e.g. "front", "enc2", "dec3", "tail"        */
    int32_t launches;    /* launches timed since the last read                         */
    float total_ms;      /* sum of their durations                                     */
} pvf_kernel_time;
PVF_API pvf_status pvf_profile_enable(pvf_handle *h, int32_t on);
/* Synchronises stream, sums the recorded durations per kernel family into out
 * (at most max_entries, *n_entries set to the number written) and clears them. */
PVF_API pvf_status pvf_profile_read(pvf_handle *h, pvf_kernel_time *out, int32_t max_entries,
                                    int32_t *n_entries, pvf_stream_t stream);

/* Steps 1-2 (validation, slice sort, FC net, histogram) in float32 without allocating any
 * device memory and without a handle or pool. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate, such as code running inside a host
 * framework that owns every device allocation and forbids new ones while events flow
 * (the fixed-pool model of a trigger), or a process whose device allocator is not
 * available to this library. The caller passes inputs and outputs only:
 *   weights_blob   host "PVFW" blob (parsed on every call; its FC layers are used)
 *   tracks         device SoA features, as for pvf_infer
 *   event_offsets  device int32[n_events + 1]
 *   n_events       0..4096 (larger: PVF_ERR_INVALID_ARG)
 *   out_hist       device float[n_events * 4000], 16-byte aligned
 *   out_bypass     device int32[n_events] or NULL: 1 where the event was bypassed (bad
 *                  offsets or more than 2048 tracks; its histogram row is all zero)
 * The kernel's scratch (the packed FC weights, 31,760 bytes, and a bypass flag per event,
 * 16,384 bytes: 48,384 bytes in all) is a fixed array inside libpvf.so that every GPU
 * loading the library holds until the process exits. The first call on each device looks
 * up that array's device address (make it before any stream capture). Every call
 * overwrites the array, which keeps the last call's contents; calls that overlap on the
 * GPU race on it. The packed weights go to the array in a copy from pageable host memory,
 * so the call may wait for work already queued on stream before it returns; the kernel
 * is then enqueued on stream and runs asynchronously. */
PVF_API pvf_status pvf_histogram_static(const void *weights_blob, size_t blob_bytes,
                                        const pvf_tracks_soa *tracks,
                                        const int32_t *event_offsets, int32_t n_events,
                                        float *out_hist, int32_t *out_bypass,
                                        pvf_stream_t stream);

/* CUDA graph of one pvf_infer launch sequence (every chunk, every kernel) for fixed
 * argument pointers: the batching form, where thousands of events run as one graph
 * launch. The graph reads the current contents of tracks, event_offsets and n_events'
 * outputs at each launch, so the caller refills those buffers between launches.
 * pvf_graph_create captures on a private stream (no work is executed) and instantiates
 * the graph; it must not be called while another capture is active on this thread.
 * Profiling (pvf_profile_enable) is suspended while capturing. */
typedef struct pvf_graph pvf_graph;
PVF_API pvf_status pvf_graph_create(pvf_handle *h, const pvf_tracks_soa *tracks,
                                    const int32_t *event_offsets, int32_t n_events,
                                    float *out_pv_z, int32_t *out_pv_count, pvf_graph **out);
/* The same with the event count read on the device at every launch: the graph covers up
 * to max_n_events events and each launch processes the first *n_events of them (clamped
 * to [0, max_n_events]), so one captured graph serves batches of any size without padding
 * them with empty events. Only the first *n_events entries of out_pv_count (and their z
 * lists) are written.
 *   n_events  int32 the device reads (device memory, or pinned host memory mapped into
 *             the device's address space), written before each launch; its value is
 *             read by the first kernel of the launch, so it may change between launches
 * Tensor-core forms (PVF_BF16, PVF_FP16, PVF_FP8_E4M3) only; PVF_FP32: UNSUPPORTED.
 * This is the batching interface of §3's fixed-shape execution with a run-time batch
 * size, as the serving loop below uses it. */
PVF_API pvf_status pvf_graph_create_dynamic(pvf_handle *h, const pvf_tracks_soa *tracks,
                                            const int32_t *event_offsets, const int32_t *n_events,
                                            int32_t max_n_events, float *out_pv_z,
                                            int32_t *out_pv_count, pvf_graph **out);
PVF_API pvf_status pvf_graph_launch(pvf_graph *g, pvf_stream_t stream);
PVF_API pvf_status pvf_graph_destroy(pvf_graph *g);

/* Serving: a continuous-batching request loop on the host (the library's runtime).
 * Requests are events of a host-side event store, arriving at given times. Whenever
 * fewer than max_inflight batches are enqueued on the stream, the loop admits the queued
 * events that fit one in-flight slot (at most max_batch events and max_tracks_per_batch
 * tracks: the slot's memory), packs their tracks into the slot's pinned staging and
 * enqueues the path on `stream`. A batch is launched as soon as a slot is free and
 * min_batch events are queued, or the oldest queued event has waited max_wait_us, or no
 * more arrivals remain.
 * Gather form (default for the tensor-core forms on a device that can map host memory):
 * before the first arrival the event store is copied into pinned host memory mapped into
 * the device's address space (events as they would land in pinned receive buffers), and
 * each slot gets one graph, captured then, that takes the batch's store indices and event
 * count from a mapped record, reads the indexed events' tracks straight from the store
 * and writes the PV counts and z lists into the record: a batch is k index writes and one
 * graph launch, with no copies and no padding.
 * Copy form (PVF_SERVE_COPY, and always for PVF_FP32): the staging is copied into the
 * caller's device_slots and the results back, around the graph of the smallest bucket of
 * 1, 2, 4, ... max_batch events that holds the batch (tracks at a fixed stride of
 * max_tracks_per_batch, missing events empty). PVF_SERVE_STREAM_LAUNCH (copy form)
 * enqueues pvf_infer instead of a graph. */
#define PVF_SERVE_STREAM_LAUNCH 1
#define PVF_SERVE_COPY 2
typedef struct {
    int32_t max_batch;            /* events per launch, 1..max_events of the handle      */
    int32_t max_tracks_per_batch; /* tracks per launch; every stored event must fit       */
    int32_t max_inflight;         /* batches enqueued at once, 1..16                      */
    int32_t min_batch;            /* >= 1                                                 */
    float max_wait_us;            /* batching window for the oldest queued event          */
    int32_t flags;                /* 0, PVF_SERVE_COPY, PVF_SERVE_COPY | STREAM_LAUNCH     */
    float launch_lead_us;         /* > 0: while a batch runs, the next one is admitted only
                                     once the running one is predicted to end within this
                                     many us (its duration from a line through the graph's
                                     times at 1 and max_batch events, measured before the
                                     first arrival), so that it takes every request that
                                     arrives meanwhile; 0: admit whenever a slot is free   */
    int32_t reserved;
} pvf_serve_config;

/* Device bytes the in-flight slots of the copy form need (inputs and outputs of
 * max_inflight batches); pvf_serve_replay requires them in every form. */
PVF_API pvf_status pvf_serve_bytes_required(const pvf_serve_config *cfg, int32_t max_pv_per_event,
                                            size_t *out_bytes);

/* Replays n_requests arrivals and blocks until every request has completed.
 *   store_f[9], store_offsets  host SoA event store (n_store events), as in pvf_infer
 *   arrival_ns[i]              host time of request i, ns after the call starts, ascending
 *   request_event[i]           store index of request i
 *   device_slots               caller-owned device memory, >= pvf_serve_bytes_required
 *   out_done_ns[i]             host time at which request i's batch was seen complete
 *   out_pv_count[i]            its PV count (-1 = bypassed), or NULL
 *   out_pv_z                   host float[n_requests * max_pv_per_event]: its z list, or NULL
 *   out_batches                number of launches, or NULL
 * Pinned host staging (one slot's size per in-flight batch) and the graphs are created
 * for the call and freed before it returns; no device memory is allocated. The graphs use
 * the handle's pool like pvf_infer, so the handle serves one call at a time. Synchronises
 * stream before returning. */
PVF_API pvf_status pvf_serve_replay(pvf_handle *h, const pvf_serve_config *cfg,
                                    const float *const *store_f, const int32_t *store_offsets,
                                    int32_t n_store, const int64_t *arrival_ns,
                                    const int32_t *request_event, int32_t n_requests,
                                    void *device_slots, size_t device_bytes, int64_t *out_done_ns,
                                    int32_t *out_pv_count, float *out_pv_z, int32_t *out_batches,
                                    pvf_stream_t stream);

/* Frees the handle's host state. The pool stays owned by the caller. NULL is a no-op. */
PVF_API pvf_status pvf_destroy(pvf_handle *h);

/* Static, never-NULL description of a status code. */
PVF_API const char *pvf_status_str(pvf_status s);

/* Library version, (major << 16) | minor. */
PVF_API int32_t pvf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PVF_H */
