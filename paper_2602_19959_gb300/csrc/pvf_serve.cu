// Continuous-batching request loop over one pvf_handle (host runtime).
//
// Requests (events) arrive at given times. Whenever fewer than max_inflight batches are
// enqueued, the loop admits the queued events that fit one slot -- at most max_batch
// events and max_tracks_per_batch tracks -- and enqueues the path for them on the single
// stream. Batches run in stream order while the host prepares the next ones, so requests
// that arrive while others are on the GPU are taken as slots free up. A CUDA event per
// slot is polled for completion; each request's completion time is the host time at
// which its batch was observed done.
//
// Gather form (the default for the tensor-core forms on a device that maps host memory):
// the event store is held in pinned host memory mapped into the device's address space
// (copied there once, before the first arrival: the model of events landing in pinned
// receive buffers), and each slot is a small mapped record -- the batch's store indices,
// its event count, and the PV counts and z lists of its results. One graph per slot
// (dynamic count, events gathered by index) reads the tracks of the indexed events
// straight from the store and writes the results into the record. A batch is thus k
// index writes, one graph launch and one event: no packing, no copy-engine transfer, and
// no padding to a bucket size.
//
// Copy form (PVF_SERVE_COPY, and the float32 form): the batch's tracks are packed into
// the slot's pinned staging and copied into the caller's device memory with one strided
// copy, the path runs as the CUDA graph of the smallest bucket (1, 2, 4, ... events, and
// max_batch) holding the batch with the missing events empty, and the counts and z lists
// are copied back. PVF_SERVE_STREAM_LAUNCH enqueues pvf_infer instead of the graphs.
#include <chrono>
#include <cstring>
#include <new>
#include <vector>

#include "pvf_internal.cuh"

namespace pvf {
namespace {

constexpr int kMaxBuckets = 16;

struct Slot {
    unsigned char *host = nullptr;   // pinned staging or record (layouts below)
    unsigned char *dev = nullptr;    // what the kernels address: the caller's device memory
                                     // (copy form) or the mapped record (gather form)
    cudaEvent_t done = nullptr;
    pvf_graph *graph[kMaxBuckets] = {};
    int r0 = 0, r1 = 0;              // requests [r0, r1) of this batch
};

// Copy form, the same layout in the staging and in device memory: feature f of the batch
// at f * MT floats, the offsets (MB + 1), then the PV counts and z lists.
struct CopyLayout {
    size_t offsets, counts, z, bytes;
    CopyLayout(int mb, int mt, int max_pv) {
        offsets = sizeof(float) * 9 * (size_t)mt;
        counts = (offsets + sizeof(int32_t) * (size_t)(mb + 1) + 255) / 256 * 256;
        z = (counts + sizeof(int32_t) * (size_t)mb + 255) / 256 * 256;
        bytes = (z + sizeof(float) * (size_t)mb * max_pv + 255) / 256 * 256;
    }
};

// Gather form, a mapped record per slot: store indices (MB), the event count, then the
// PV counts and z lists.
struct GatherLayout {
    size_t index = 0, count, counts, z, bytes;
    GatherLayout(int mb, int max_pv) {
        count = sizeof(int32_t) * (size_t)mb;
        counts = (count + sizeof(int32_t) + 255) / 256 * 256;
        z = (counts + sizeof(int32_t) * (size_t)mb + 255) / 256 * 256;
        bytes = (z + sizeof(float) * (size_t)mb * max_pv + 255) / 256 * 256;
    }
};

}  // namespace
}  // namespace pvf

using namespace pvf;

extern "C" {

pvf_status pvf_serve_bytes_required(const pvf_serve_config *cfg, int32_t max_pv_per_event,
                                    size_t *out) {
    if (!cfg || !out || cfg->max_batch < 1 || cfg->max_inflight < 1 || cfg->max_inflight > 16 ||
        cfg->max_tracks_per_batch < 1 || max_pv_per_event < 1)
        return PVF_ERR_INVALID_ARG;
    *out = (size_t)cfg->max_inflight * CopyLayout(cfg->max_batch, cfg->max_tracks_per_batch, max_pv_per_event).bytes;
    return PVF_OK;
}

pvf_status pvf_serve_replay(pvf_handle *h, const pvf_serve_config *cfg, const float *const *store_f,
                            const int32_t *store_offsets, int32_t n_store, const int64_t *arrival_ns,
                            const int32_t *request_event, int32_t n_requests, void *device_slots,
                            size_t device_bytes, int64_t *out_done_ns, int32_t *out_pv_count,
                            float *out_pv_z, int32_t *out_batches, pvf_stream_t stream_) {
    if (!h || !cfg || !store_f || !store_offsets || n_store < 1 || !arrival_ns || !request_event ||
        n_requests < 0 || !device_slots || !out_done_ns)
        return PVF_ERR_INVALID_ARG;
    for (int k = 0; k < 9; ++k) if (!store_f[k]) return PVF_ERR_INVALID_ARG;
    const int max_pv = pvf_handle_max_pv(h), max_events = pvf_handle_max_events(h);
    if (cfg->max_batch < 1 || cfg->max_batch > max_events || cfg->max_inflight < 1 ||
        cfg->max_inflight > 16 || cfg->max_tracks_per_batch < 1 || cfg->min_batch < 1 ||
        (cfg->flags & ~(PVF_SERVE_STREAM_LAUNCH | PVF_SERVE_COPY)))
        return PVF_ERR_INVALID_ARG;
    size_t need = 0;
    if (pvf_serve_bytes_required(cfg, max_pv, &need) != PVF_OK || device_bytes < need)
        return PVF_ERR_POOL_TOO_SMALL;
    if (store_offsets[0] != 0) return PVF_ERR_INVALID_ARG;
    for (int e = 0; e < n_store; ++e)
        if (store_offsets[e + 1] < store_offsets[e]) return PVF_ERR_INVALID_ARG;
    for (int i = 0; i < n_requests; ++i) {
        const int ev = request_event[i];
        if (ev < 0 || ev >= n_store || (i && arrival_ns[i] < arrival_ns[i - 1])) return PVF_ERR_INVALID_ARG;
        const int nt = store_offsets[ev + 1] - store_offsets[ev];
        if (nt > cfg->max_tracks_per_batch) return PVF_ERR_INVALID_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    const int MB = cfg->max_batch, MT = cfg->max_tracks_per_batch;
    const int64_t n_store_tracks = store_offsets[n_store];
    const bool stream_launch = (cfg->flags & PVF_SERVE_STREAM_LAUNCH) != 0;
    int dev = 0, can_map = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&can_map, cudaDevAttrCanMapHostMemory, dev) != cudaSuccess)
        return PVF_ERR_CUDA;
    const bool gather = !stream_launch && !(cfg->flags & PVF_SERVE_COPY) && can_map &&
                        pvf_handle_precision(h) != PVF_FP32;
    const CopyLayout cl(MB, MT, max_pv);
    const GatherLayout gl(MB, max_pv);
    const size_t off_counts = gather ? gl.counts : cl.counts, off_z = gather ? gl.z : cl.z;

    std::vector<Slot> slots(cfg->max_inflight);
    std::vector<int> buckets;            // copy form: 1, 2, 4, ... < MB, then MB
    if (!gather) {
        for (int b = 1; b < MB; b *= 2) buckets.push_back(b);
        buckets.push_back(MB);
        if ((int)buckets.size() > kMaxBuckets) return PVF_ERR_INVALID_ARG;
    }
    pvf_status st = PVF_OK;
    // gather form: the store in mapped pinned memory, features [9][n] then the offsets
    unsigned char *store_h = nullptr, *store_d = nullptr;
    pvf_tracks_soa store_tr{};
    const int32_t *store_off_d = nullptr;
    if (gather) {
        const size_t fbytes = sizeof(float) * (size_t)n_store_tracks;
        const size_t bytes = 9 * fbytes + sizeof(int32_t) * (size_t)(n_store + 1) + 16;
        void *p = nullptr;
        if (cudaHostAlloc(&store_h, bytes, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer(&p, store_h, 0) != cudaSuccess) {
            st = PVF_ERR_CUDA;
        } else {
            store_d = static_cast<unsigned char *>(p);
            for (int f = 0; f < 9; ++f) {
                std::memcpy(store_h + f * fbytes, store_f[f], fbytes);
                store_tr.f[f] = reinterpret_cast<const float *>(store_d + f * fbytes);
            }
            store_tr.n_tracks = n_store_tracks;
            std::memcpy(store_h + 9 * fbytes, store_offsets, sizeof(int32_t) * (size_t)(n_store + 1));
            store_off_d = reinterpret_cast<const int32_t *>(store_d + 9 * fbytes);
        }
    }
    auto slot_tracks = [&](const Slot &sl) {
        pvf_tracks_soa tr;
        float *df = reinterpret_cast<float *>(sl.dev);
        for (int f = 0; f < 9; ++f) tr.f[f] = df + (size_t)f * MT;
        tr.n_tracks = MT;
        return tr;
    };
    for (size_t i = 0; i < slots.size() && st == PVF_OK; ++i) {
        Slot &sl = slots[i];
        if (cudaHostAlloc(&sl.host, gather ? gl.bytes : cl.bytes,
                          gather ? cudaHostAllocMapped : cudaHostAllocDefault) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            st = PVF_ERR_CUDA;
            break;
        }
        if (gather) {
            void *p = nullptr;
            if (cudaHostGetDevicePointer(&p, sl.host, 0) != cudaSuccess) { st = PVF_ERR_CUDA; break; }
            sl.dev = static_cast<unsigned char *>(p);
            st = graph_create_gather(h, &store_tr, store_off_d, reinterpret_cast<int32_t *>(sl.dev + gl.index),
                                     reinterpret_cast<int32_t *>(sl.dev + gl.count), MB,
                                     reinterpret_cast<float *>(sl.dev + gl.z),
                                     reinterpret_cast<int32_t *>(sl.dev + gl.counts), &sl.graph[0]);
            continue;
        }
        sl.dev = static_cast<unsigned char *>(device_slots) + i * cl.bytes;
        if (stream_launch) continue;
        const pvf_tracks_soa tr = slot_tracks(sl);
        int32_t *doff = reinterpret_cast<int32_t *>(sl.dev + cl.offsets);
        int32_t *dcnt = reinterpret_cast<int32_t *>(sl.dev + cl.counts);
        float *dz = reinterpret_cast<float *>(sl.dev + cl.z);
        for (size_t b = 0; b < buckets.size() && st == PVF_OK; ++b)
            st = pvf_graph_create(h, &tr, doff, buckets[b], dz, dcnt, &sl.graph[b]);
    }
    // launch timing (gather form): the device time of a batch of k events, on a line
    // through the times measured here at 1 and MB events (store events 0, 1, ...)
    double t_one_ns = 0.0, t_mb_ns = 0.0;
    const bool lead = gather && cfg->launch_lead_us > 0.0f && st == PVF_OK;
    if (lead) {
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (cudaEventCreate(&ea) != cudaSuccess || cudaEventCreate(&eb) != cudaSuccess) st = PVF_ERR_CUDA;
        for (int rep = 0; rep < 4 && st == PVF_OK; ++rep)
            for (int which = 0; which < 2 && st == PVF_OK; ++which) {
                const int k = which ? MB : 1;
                Slot &sl = slots[0];
                int32_t *idx = reinterpret_cast<int32_t *>(sl.host + gl.index);
                for (int i = 0; i < k; ++i) idx[i] = i % n_store;
                *reinterpret_cast<volatile int32_t *>(sl.host + gl.count) = k;
                float ms = 0.0f;
                if (cudaEventRecord(ea, s) != cudaSuccess || pvf_graph_launch(sl.graph[0], stream_) != PVF_OK ||
                    cudaEventRecord(eb, s) != cudaSuccess || cudaEventSynchronize(eb) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, ea, eb) != cudaSuccess) {
                    st = PVF_ERR_CUDA;
                    break;
                }
                if (rep == 0) continue;                      // the first launch warms up
                double &t = which ? t_mb_ns : t_one_ns;
                if (t == 0.0 || ms * 1e6 < t) t = ms * 1e6;   // fastest of three
            }
        if (ea) cudaEventDestroy(ea);
        if (eb) cudaEventDestroy(eb);
    }
    auto predict_ns = [&](int k) {
        return t_one_ns + (t_mb_ns - t_one_ns) * (double)(k - 1) / (double)(MB > 1 ? MB - 1 : 1);
    };
    const double lead_ns = 1000.0 * cfg->launch_lead_us;
    double end_est = 0.0;              // predicted end (host ns) of the last enqueued batch
    std::vector<int32_t> batch_offsets(MB + 1);
    using clock = std::chrono::steady_clock;
    const auto t_start = clock::now();
    auto now_ns = [&]() {
        return (int64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(clock::now() - t_start).count();
    };
    int next_arr = 0, q_head = 0, completed = 0, batches = 0, ring_head = 0, ring_n = 0;
    const int nslots = (int)slots.size();
    while (st == PVF_OK && completed < n_requests) {
        const int64_t now = now_ns();
        while (next_arr < n_requests && arrival_ns[next_arr] <= now) ++next_arr;
        // completions, in stream order
        while (ring_n > 0) {
            Slot &sl = slots[ring_head];
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) { st = PVF_ERR_CUDA; break; }
            const int64_t t_done = now_ns();
            const int32_t *cnt = reinterpret_cast<const int32_t *>(sl.host + off_counts);
            const float *zz = reinterpret_cast<const float *>(sl.host + off_z);
            for (int r = sl.r0; r < sl.r1; ++r) {
                out_done_ns[r] = t_done;
                const int c = cnt[r - sl.r0];
                if (out_pv_count) out_pv_count[r] = c;
                if (out_pv_z && c > 0)
                    std::memcpy(out_pv_z + (size_t)r * max_pv, zz + (size_t)(r - sl.r0) * max_pv,
                                sizeof(float) * (size_t)(c < max_pv ? c : max_pv));
            }
            completed += sl.r1 - sl.r0;
            ring_head = (ring_head + 1) % nslots;
            --ring_n;
        }
        if (st != PVF_OK) break;
        // admission: a free slot and queued requests (and, with a launch lead, the running
        // batch about to end, so that the next one takes everything that arrives before)
        const int queued = next_arr - q_head;
        const bool due = !lead || ring_n == 0 || end_est - (double)now <= lead_ns;
        if (ring_n < nslots && queued > 0 && due) {
            const bool all_arrived = next_arr == n_requests;
            const bool waited = (double)(now - arrival_ns[q_head]) >= 1000.0 * cfg->max_wait_us;
            if (queued >= cfg->min_batch || waited || all_arrived) {
                Slot &sl = slots[(ring_head + ring_n) % nslots];
                int r = q_head, ntr = 0, k = 0;
                batch_offsets[0] = 0;
                while (r < next_arr && k < MB) {
                    const int ev = request_event[r];
                    const int nt = store_offsets[ev + 1] - store_offsets[ev];
                    if (ntr + nt > MT) break;
                    ntr += nt;
                    batch_offsets[++k] = ntr;
                    ++r;
                }
                bool ok = true;
                if (gather) {
                    int32_t *idx = reinterpret_cast<int32_t *>(sl.host + gl.index);
                    std::memcpy(idx, request_event + q_head, sizeof(int32_t) * k);
                    *reinterpret_cast<volatile int32_t *>(sl.host + gl.count) = k;
                    ok = pvf_graph_launch(sl.graph[0], stream_) == PVF_OK;
                } else {
                    size_t bi = 0;
                    while (!stream_launch && buckets[bi] < k) ++bi;
                    // events launched: the bucket's size with the missing events empty
                    const int kb = stream_launch ? k : buckets[bi];
                    for (int i = k + 1; i <= kb; ++i) batch_offsets[i] = ntr;
                    // pack feature f of the batch at f * MT floats, then the offsets
                    float *hf = reinterpret_cast<float *>(sl.host);
                    for (int f = 0; f < 9; ++f) {
                        float *dst = hf + (size_t)f * MT;
                        for (int i = 0; i < k; ++i) {
                            const int ev = request_event[q_head + i];
                            const int a = store_offsets[ev], nt = store_offsets[ev + 1] - a;
                            std::memcpy(dst + batch_offsets[i], store_f[f] + a, sizeof(float) * nt);
                        }
                    }
                    int32_t *ho = reinterpret_cast<int32_t *>(sl.host + cl.offsets);
                    std::memcpy(ho, batch_offsets.data(), sizeof(int32_t) * (kb + 1));
                    const pvf_tracks_soa tr = slot_tracks(sl);
                    int32_t *doff = reinterpret_cast<int32_t *>(sl.dev + cl.offsets);
                    int32_t *dcnt = reinterpret_cast<int32_t *>(sl.dev + cl.counts);
                    float *dz = reinterpret_cast<float *>(sl.dev + cl.z);
                    if (ntr > 0)   // the batch's tracks of each feature row, one strided copy
                        ok = cudaMemcpy2DAsync(sl.dev, sizeof(float) * MT, sl.host, sizeof(float) * MT,
                                               sizeof(float) * ntr, 9, cudaMemcpyHostToDevice, s) == cudaSuccess;
                    ok = ok && cudaMemcpyAsync(doff, ho, sizeof(int32_t) * (kb + 1), cudaMemcpyHostToDevice,
                                               s) == cudaSuccess;
                    if (ok) {
                        ok = !stream_launch ? pvf_graph_launch(sl.graph[bi], stream_) == PVF_OK
                                            : pvf_infer(h, &tr, doff, k, dz, dcnt, stream_) == PVF_OK;
                    }
                    ok = ok &&
                         cudaMemcpyAsync(sl.host + cl.counts, dcnt, sizeof(int32_t) * k, cudaMemcpyDeviceToHost,
                                         s) == cudaSuccess &&
                         cudaMemcpyAsync(sl.host + cl.z, dz, sizeof(float) * (size_t)k * max_pv,
                                         cudaMemcpyDeviceToHost, s) == cudaSuccess;
                }
                ok = ok && cudaEventRecord(sl.done, s) == cudaSuccess;
                if (!ok) {
                    st = PVF_ERR_CUDA;
                    break;
                }
                sl.r0 = q_head;
                sl.r1 = q_head + k;
                if (lead) end_est = (ring_n == 0 || end_est < (double)now ? (double)now : end_est) + predict_ns(k);
                ++ring_n;
                ++batches;
                q_head += k;
            }
        }
    }
    // nothing may still read or write the pinned memory when it is freed
    if (cudaStreamSynchronize(s) != cudaSuccess && st == PVF_OK) st = PVF_ERR_CUDA;
    for (auto &sl : slots) {
        for (int b = 0; b < kMaxBuckets; ++b) pvf_graph_destroy(sl.graph[b]);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.host) cudaFreeHost(sl.host);
    }
    if (store_h) cudaFreeHost(store_h);
    if (out_batches) *out_batches = batches;
    return st;
}

}  // extern "C"
