// Continuous-batching request loop over one pvf_handle (host runtime).
//
// Requests (events) arrive at given times. Whenever fewer than max_inflight batches are
// enqueued, the loop admits the queued events that fit one slot -- at most max_batch
// events and max_tracks_per_batch tracks, the slot's share of the caller's device
// memory -- packs their Structure-of-Arrays tracks into the slot's pinned staging
// buffer, and enqueues on the single stream: the host->device copies, the path, and the
// copies of the PV counts and z lists back. Batches run in stream order while the host
// packs the next ones, so requests that arrive while others are on the GPU are taken as
// slots free up. A CUDA event per slot is polled for completion; each request's
// completion time is the host time at which its batch was observed done.
//
// The path runs as a CUDA graph per (slot, bucket): the slot's tracks sit at a fixed
// stride of max_tracks_per_batch floats per feature, so one graph of B events serves
// every batch of k <= B events (offsets k+1..B repeat the track count: empty events).
// Buckets are 1, 2, 4, ... and max_batch; the graphs are captured before the clock starts.
#include <chrono>
#include <cstring>
#include <new>
#include <vector>

#include "pvf_internal.cuh"

namespace pvf {
namespace {

constexpr int kMaxBuckets = 16;

struct Slot {
    unsigned char *host = nullptr;   // pinned: [9][MT] features | offsets | counts | z
    unsigned char *dev = nullptr;    // caller's device memory, same layout
    cudaEvent_t done = nullptr;
    pvf_graph *graph[kMaxBuckets] = {};
    int r0 = 0, r1 = 0;              // requests [r0, r1) of this batch
    int nt = 0;                      // tracks packed
    bool busy = false;
};

size_t slot_bytes(int max_batch, int max_tracks, int max_pv) {
    size_t b = sizeof(float) * 9 * (size_t)max_tracks + sizeof(int32_t) * (size_t)(max_batch + 1);
    b = (b + 255) / 256 * 256;
    b += sizeof(int32_t) * (size_t)max_batch;
    b = (b + 255) / 256 * 256;
    b += sizeof(float) * (size_t)max_batch * max_pv;
    return (b + 255) / 256 * 256;
}

}  // namespace
}  // namespace pvf

using namespace pvf;

extern "C" {

pvf_status pvf_serve_bytes_required(const pvf_serve_config *cfg, int32_t max_pv_per_event,
                                    size_t *out) {
    if (!cfg || !out || cfg->max_batch < 1 || cfg->max_inflight < 1 || cfg->max_inflight > 16 ||
        cfg->max_tracks_per_batch < 1 || max_pv_per_event < 1)
        return PVF_ERR_INVALID_ARG;
    *out = (size_t)cfg->max_inflight * slot_bytes(cfg->max_batch, cfg->max_tracks_per_batch, max_pv_per_event);
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
        cfg->max_inflight > 16 || cfg->max_tracks_per_batch < 1 || cfg->min_batch < 1)
        return PVF_ERR_INVALID_ARG;
    size_t need = 0;
    if (pvf_serve_bytes_required(cfg, max_pv, &need) != PVF_OK || device_bytes < need)
        return PVF_ERR_POOL_TOO_SMALL;
    for (int i = 0; i < n_requests; ++i) {
        const int ev = request_event[i];
        if (ev < 0 || ev >= n_store || (i && arrival_ns[i] < arrival_ns[i - 1])) return PVF_ERR_INVALID_ARG;
        const int nt = store_offsets[ev + 1] - store_offsets[ev];
        if (nt < 0 || nt > cfg->max_tracks_per_batch) return PVF_ERR_INVALID_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    const int MB = cfg->max_batch, MT = cfg->max_tracks_per_batch;
    const size_t sb = slot_bytes(MB, MT, max_pv);
    const size_t off_counts = ((sizeof(float) * 9 * (size_t)MT + sizeof(int32_t) * (MB + 1)) + 255) / 256 * 256;
    const size_t off_z = (off_counts + sizeof(int32_t) * MB + 255) / 256 * 256;

    std::vector<Slot> slots(cfg->max_inflight);
    const bool use_graphs = !(cfg->flags & PVF_SERVE_STREAM_LAUNCH);
    std::vector<int> buckets;            // 1, 2, 4, ... < MB, then MB
    for (int b = 1; b < MB; b *= 2) buckets.push_back(b);
    buckets.push_back(MB);
    if ((int)buckets.size() > kMaxBuckets) return PVF_ERR_INVALID_ARG;
    // fixed layout of a slot: feature f at f * MT floats, then the offsets
    auto slot_tracks = [&](const Slot &sl) {
        pvf_tracks_soa tr;
        float *df = reinterpret_cast<float *>(sl.dev);
        for (int f = 0; f < 9; ++f) tr.f[f] = df + (size_t)f * MT;
        tr.n_tracks = MT;
        return tr;
    };
    const size_t off_offsets = sizeof(float) * 9 * (size_t)MT;
    pvf_status st = PVF_OK;
    for (size_t i = 0; i < slots.size() && st == PVF_OK; ++i) {
        Slot &sl = slots[i];
        sl.dev = static_cast<unsigned char *>(device_slots) + i * sb;
        if (cudaHostAlloc(&sl.host, sb, cudaHostAllocDefault) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            st = PVF_ERR_CUDA;
            break;
        }
        if (use_graphs) {
            const pvf_tracks_soa tr = slot_tracks(sl);
            int32_t *doff = reinterpret_cast<int32_t *>(sl.dev + off_offsets);
            int32_t *dcnt = reinterpret_cast<int32_t *>(sl.dev + off_counts);
            float *dz = reinterpret_cast<float *>(sl.dev + off_z);
            for (size_t b = 0; b < buckets.size() && st == PVF_OK; ++b)
                st = pvf_graph_create(h, &tr, doff, buckets[b], dz, dcnt, &sl.graph[b]);
        }
    }
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
                if (out_pv_count) out_pv_count[r] = cnt[r - sl.r0];
                if (out_pv_z)
                    std::memcpy(out_pv_z + (size_t)r * max_pv, zz + (size_t)(r - sl.r0) * max_pv,
                                sizeof(float) * max_pv);
            }
            completed += sl.r1 - sl.r0;
            sl.busy = false;
            ring_head = (ring_head + 1) % nslots;
            --ring_n;
        }
        if (st != PVF_OK) break;
        // admission: a free slot and queued requests
        const int queued = next_arr - q_head;
        if (ring_n < nslots && queued > 0) {
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
                size_t bi = 0;
                while (use_graphs && buckets[bi] < k) ++bi;
                const int kb = use_graphs ? buckets[bi] : k;     // events launched
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
                int32_t *ho = reinterpret_cast<int32_t *>(sl.host + off_offsets);
                std::memcpy(ho, batch_offsets.data(), sizeof(int32_t) * (kb + 1));
                const pvf_tracks_soa tr = slot_tracks(sl);
                int32_t *doff = reinterpret_cast<int32_t *>(sl.dev + off_offsets);
                int32_t *dcnt = reinterpret_cast<int32_t *>(sl.dev + off_counts);
                float *dz = reinterpret_cast<float *>(sl.dev + off_z);
                bool ok = true;
                if (ntr > 0)   // the batch's tracks of each feature row, one strided copy
                    ok = cudaMemcpy2DAsync(sl.dev, sizeof(float) * MT, sl.host, sizeof(float) * MT,
                                           sizeof(float) * ntr, 9, cudaMemcpyHostToDevice, s) == cudaSuccess;
                ok = ok && cudaMemcpyAsync(doff, ho, sizeof(int32_t) * (kb + 1), cudaMemcpyHostToDevice,
                                           s) == cudaSuccess;
                if (ok) {
                    ok = use_graphs ? pvf_graph_launch(sl.graph[bi], stream_) == PVF_OK
                                    : pvf_infer(h, &tr, doff, k, dz, dcnt, stream_) == PVF_OK;
                }
                ok = ok &&
                     cudaMemcpyAsync(sl.host + off_counts, dcnt, sizeof(int32_t) * k, cudaMemcpyDeviceToHost,
                                     s) == cudaSuccess &&
                     cudaMemcpyAsync(sl.host + off_z, dz, sizeof(float) * (size_t)k * max_pv,
                                     cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                     cudaEventRecord(sl.done, s) == cudaSuccess;
                if (!ok) {
                    st = PVF_ERR_CUDA;
                    break;
                }
                sl.r0 = q_head;
                sl.r1 = q_head + k;
                sl.nt = ntr;
                sl.busy = true;
                ++ring_n;
                ++batches;
                q_head += k;
            }
        }
    }
    if (st != PVF_OK) cudaStreamSynchronize(s);
    for (auto &sl : slots) {
        for (int b = 0; b < kMaxBuckets; ++b) pvf_graph_destroy(sl.graph[b]);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.host) cudaFreeHost(sl.host);
    }
    if (out_batches) *out_batches = batches;
    return st;
}

}  // extern "C"
