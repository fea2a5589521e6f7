// C ABI of libpvf (declared in include/pvf.h): argument validation, the weight blob
// reader, the pool plan and the launch sequence of one pvf_infer call.
//
// The translation layer of the paper (§3: Prepare / Execute / Extract) reduces here to
// host-side validation and pointer arithmetic: the caller's Structure-of-Arrays
// features are read in place by the first kernel, every intermediate lives at a fixed
// offset of the caller's pool, and every launch goes to the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pvf_internal.cuh"
#include "pvf_tc.cuh"

namespace pvf {
namespace {

constexpr uint32_t kBlobVersion = 1;
constexpr int kNumLayers = 17;
const char *const kLayerNames[kNumLayers] = {"fc1", "fc2", "fc3", "fc4", "fc5", "fc6",
                                             "enc1", "enc2", "enc3", "enc4", "up3", "dec3",
                                             "up2", "dec2", "up1", "dec1", "final"};

struct BlobHeader {
    char magic[4];
    uint32_t version, c0, fc_hidden, fc_out, n_layers, reserved[2];
};
struct LayerEntry {
    char name[8];
    uint32_t ndim, shape[3], n_bias, pad;
    uint64_t w_offset, b_offset;
};
static_assert(sizeof(BlobHeader) == 32 && sizeof(LayerEntry) == 48, "blob layout");

struct HostLayer {
    std::vector<float> w, b;
    uint32_t shape[3];
};

// Expected (weight shape, bias length) of layer i for the supported architecture with
// UNet base width c0 (16, or 32 for the wide float32 variant).
void expected_shape(int i, int c0, uint32_t shape[3], uint32_t *nb) {
    const uint32_t h = kFcHidden, c1 = c0, c2 = 2 * c0, c3 = 4 * c0, c4 = 8 * c0;
    const uint32_t tbl[kNumLayers][4] = {          // built per call: it depends on c0
        {h, 9, 0, h}, {h, h, 0, h}, {h, h, 0, h}, {h, h, 0, h}, {h, h, 0, h}, {100, h, 0, 100},
        {c1, 1, 5, c1}, {c2, c1, 5, c2}, {c3, c2, 5, c3}, {c4, c3, 5, c4},
        {c4, c3, 2, c3}, {c3, 2 * c3, 5, c3}, {c3, c2, 2, c2}, {c2, 2 * c2, 5, c2},
        {c2, c1, 2, c1}, {c1, 2 * c1, 5, c1}, {1, c1, 5, 1}};
    shape[0] = tbl[i][0];
    shape[1] = tbl[i][1];
    shape[2] = tbl[i][2];
    *nb = tbl[i][3];
}

// c0: the base width the blob must have (0: either supported width, returned in *c0_out).
pvf_status parse_blob(const void *blob, size_t bytes, int c0, std::vector<HostLayer> &layers,
                      int *c0_out = nullptr) {
    if (!blob || bytes < sizeof(BlobHeader)) return PVF_ERR_WEIGHTS;
    BlobHeader hd;
    std::memcpy(&hd, blob, sizeof hd);
    if (hd.c0 != (uint32_t)kC0 && hd.c0 != (uint32_t)kC0Max) return PVF_ERR_WEIGHTS;
    if (c0 && hd.c0 != (uint32_t)c0) return PVF_ERR_WEIGHTS;
    c0 = (int)hd.c0;
    if (c0_out) *c0_out = c0;
    if (std::memcmp(hd.magic, "PVFW", 4) != 0 || hd.version != kBlobVersion ||
        hd.fc_hidden != (uint32_t)kFcHidden || hd.fc_out != (uint32_t)kFcOut ||
        hd.n_layers != (uint32_t)kNumLayers)
        return PVF_ERR_WEIGHTS;
    if (bytes < sizeof(BlobHeader) + kNumLayers * sizeof(LayerEntry)) return PVF_ERR_WEIGHTS;
    layers.assign(kNumLayers, HostLayer());
    const unsigned char *base = static_cast<const unsigned char *>(blob);
    for (int i = 0; i < kNumLayers; ++i) {
        LayerEntry le;
        std::memcpy(&le, base + sizeof(BlobHeader) + i * sizeof(LayerEntry), sizeof le);
        if (strncmp(le.name, kLayerNames[i], 8) != 0) return PVF_ERR_WEIGHTS;
        uint32_t shp[3], nb;
        expected_shape(i, c0, shp, &nb);
        const uint32_t ndim = shp[2] ? 3 : 2;
        if (le.ndim != ndim || le.shape[0] != shp[0] || le.shape[1] != shp[1] ||
            (ndim == 3 && le.shape[2] != shp[2]) || le.n_bias != nb)
            return PVF_ERR_WEIGHTS;
        const uint64_t nw = (uint64_t)shp[0] * shp[1] * (ndim == 3 ? shp[2] : 1);
        if (le.w_offset % 4 || le.b_offset % 4 || le.w_offset > bytes ||
            nw * 4 > bytes - le.w_offset || le.b_offset > bytes || (uint64_t)nb * 4 > bytes - le.b_offset)
            return PVF_ERR_WEIGHTS;
        HostLayer &L = layers[i];
        L.w.resize(nw);
        L.b.resize(nb);
        std::memcpy(L.w.data(), base + le.w_offset, nw * 4);
        std::memcpy(L.b.data(), base + le.b_offset, (size_t)nb * 4);
        for (float v : L.w) if (!std::isfinite(v)) return PVF_ERR_WEIGHTS;
        for (float v : L.b) if (!std::isfinite(v)) return PVF_ERR_WEIGHTS;
        std::memcpy(L.shape, shp, sizeof shp);
    }
    return PVF_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

size_t elem_bytes(int precision) {
    return precision == PVF_FP32 ? 4 : is16(precision) ? 2 : 1;
}

// Float32 weight block: FC, enc1, final, conv and ConvT layers in CUDA-core layouts.
struct F32Layout {
    size_t fc, enc1, fin, conv_w[6], conv_b[6], up_w[3], up_b[3], total;  // float offsets
};
const int kConvLayer[6] = {7, 8, 9, 11, 13, 15};    // enc2, enc3, enc4, dec3, dec2, dec1
const int kUpLayer[3] = {10, 12, 14};               // up3, up2, up1

F32Layout f32_layout(int c0) {
    F32Layout L{};
    size_t o = 0;
    auto take = [&](size_t n) { size_t r = o; o += (n + 63) / 64 * 64; return r; };
    L.fc = take(kFcFloats);
    L.enc1 = take(6 * (size_t)c0);
    L.fin = take(5 * (size_t)c0 + 1);
    uint32_t shp[3], nb;
    for (int k = 0; k < 6; ++k) {
        expected_shape(kConvLayer[k], c0, shp, &nb);
        L.conv_w[k] = take((size_t)shp[0] * shp[1] * 5);
        L.conv_b[k] = take(nb);
    }
    for (int k = 0; k < 3; ++k) {
        expected_shape(kUpLayer[k], c0, shp, &nb);
        L.up_w[k] = take((size_t)shp[0] * shp[1] * 2);
        L.up_b[k] = take(nb);
    }
    L.total = o;
    return L;
}

void fill_f32(const std::vector<HostLayer> &Ls, const F32Layout &L, int c0, std::vector<float> &out) {
    out.assign(L.total, 0.0f);
    float *fc = out.data() + L.fc;
    for (int l = 0; l < 6; ++l) {
        const HostLayer &H = Ls[l];
        const int nout = H.shape[0], nin = H.shape[1];
        const int pitch = l == 0 ? kFcInPad : kFcHidden;
        for (int o = 0; o < nout; ++o)
            for (int i = 0; i < nin; ++i) {
                const float w = H.w[(size_t)o * nin + i];
                if (l < 5) fc[fc_w_off(l) + o * pitch + i] = w;
                else fc[fc_w_off(l) + i * kFcOut + o] = w;      // layer 6 transposed
            }
        for (int o = 0; o < nout; ++o) fc[fc_b_off(l) + o] = H.b[o];
    }
    {   // enc1 W[co][0][t] -> [t][co]
        const HostLayer &H = Ls[6];
        float *d = out.data() + L.enc1;
        for (int co = 0; co < c0; ++co)
            for (int t = 0; t < 5; ++t) d[t * c0 + co] = H.w[(size_t)co * 5 + t];
        for (int co = 0; co < c0; ++co) d[5 * c0 + co] = H.b[co];
    }
    {   // final W[0][ci][t] -> [t][ci]
        const HostLayer &H = Ls[16];
        float *d = out.data() + L.fin;
        for (int ci = 0; ci < c0; ++ci)
            for (int t = 0; t < 5; ++t) d[t * c0 + ci] = H.w[(size_t)ci * 5 + t];
        d[5 * c0] = H.b[0];
    }
    for (int k = 0; k < 6; ++k) {   // conv W[co][ci][t] -> [t][ci][co]
        const HostLayer &H = Ls[kConvLayer[k]];
        const int cout = H.shape[0], cin = H.shape[1];
        float *d = out.data() + L.conv_w[k];
        for (int co = 0; co < cout; ++co)
            for (int ci = 0; ci < cin; ++ci)
                for (int t = 0; t < 5; ++t)
                    d[((size_t)t * cin + ci) * cout + co] = H.w[((size_t)co * cin + ci) * 5 + t];
        std::memcpy(out.data() + L.conv_b[k], H.b.data(), sizeof(float) * cout);
    }
    for (int k = 0; k < 3; ++k) {   // ConvT W[ci][co][r] -> [ci][r][co]
        const HostLayer &H = Ls[kUpLayer[k]];
        const int cin = H.shape[0], cout = H.shape[1];
        float *d = out.data() + L.up_w[k];
        for (int ci = 0; ci < cin; ++ci)
            for (int co = 0; co < cout; ++co)
                for (int r = 0; r < 2; ++r)
                    d[((size_t)ci * 2 + r) * cout + co] = H.w[((size_t)ci * cout + co) * 2 + r];
        std::memcpy(out.data() + L.up_b[k], H.b.data(), sizeof(float) * cout);
    }
}

struct Plan {
    size_t status, ev_flag, f32w, tcw, logits, act, total;
    size_t act_slot_big, act_slot_small;   // bytes per slot for the chunk
    int chunk;
};

pvf_status check_config(const pvf_config *c) {
    if (!c) return PVF_ERR_INVALID_ARG;
    if (c->precision < PVF_FP32 || c->precision > PVF_FP16) return PVF_ERR_INVALID_ARG;
    if (c->max_events < 1 || c->max_events > (1 << 24)) return PVF_ERR_INVALID_ARG;
    if (c->max_tracks_per_event < 1 || c->max_tracks_per_event > 8192) return PVF_ERR_INVALID_ARG;
    if (c->max_pv_per_event < 1 || c->max_pv_per_event > 1024) return PVF_ERR_INVALID_ARG;
    if (c->chunk_events < 0 || c->chunk_events > c->max_events) return PVF_ERR_INVALID_ARG;
    if (!(c->boundary_mm >= 0.0f && c->boundary_mm < 5.0f)) return PVF_ERR_INVALID_ARG;
    if (c->unet_width != 0 && c->unet_width != kC0 && c->unet_width != kC0Max) return PVF_ERR_INVALID_ARG;
    if (c->per_interval != 0 && c->per_interval != 1) return PVF_ERR_INVALID_ARG;
    if (c->per_interval && c->unet_width == kC0Max) return PVF_ERR_UNSUPPORTED;
    if (c->schedule) {
        const pvf_schedule &q = *c->schedule;
        if (q.front_ctas_per_sm < 0 || q.tail_ctas_per_sm < 0) return PVF_ERR_INVALID_ARG;
        for (int k = 0; k < 6; ++k) if (q.conv_ctas_per_sm[k] < 0) return PVF_ERR_INVALID_ARG;
    }
    return PVF_OK;
}

int cfg_c0(const pvf_config *c) { return c->unet_width ? c->unet_width : kC0; }

// Largest per-event (L + 4) * C over the tensors of the big slots (e1..e4, u1..u3, d1..d3)
// and of the small ones (p1..p3), for sequences of L0 bins, base width c0, seqs per event.
void slot_elems(int L0, int c0, int seqs, size_t *big, size_t *small) {
    auto rows = [](int L) { return (size_t)(L + 2 * kPad); };
    size_t b = 0, s = 0;
    for (int k = 0; k < 4; ++k) b = std::max(b, rows(L0 >> k) * ((size_t)c0 << k));
    for (int k = 1; k < 4; ++k) s = std::max(s, rows(L0 >> k) * ((size_t)c0 << (k - 1)));
    *big = b * seqs;
    *small = s * seqs;
}

constexpr int kMaxIvChunk = 65535 / kSlices;
// Byte offsets, inside the 256-byte status block, of the front's event ticket and of the
// device copy of a dynamic event count (status word at 0, calibration maxima at 64, tile
// schedulers at 128..176).
constexpr size_t kFrontCtrOff = 176;
constexpr size_t kDynCountOff = 192;

Plan make_plan(const pvf_config *c) {
    Plan p{};
    p.chunk = c->chunk_events ? c->chunk_events : c->max_events;
    // per-interval layout: one grid row per sequence, kSlices per event (at most 65535)
    if (c->per_interval && p.chunk > kMaxIvChunk) p.chunk = kMaxIvChunk;
    size_t o = 0;
    p.status = o; o += 256;
    p.ev_flag = o; o = align256(o + sizeof(int32_t) * (size_t)c->max_events);
    const int c0 = cfg_c0(c);
    p.f32w = o; o = align256(o + sizeof(float) * f32_layout(c0).total);
    p.tcw = o; o = align256(o + tc_weight_bytes(c->precision, c0));
    p.logits = o; o = align256(o + (c->precision != PVF_FP32 ? sizeof(float) * kBins * (size_t)p.chunk : 0));
    const size_t eb = elem_bytes(c->precision);
    // every activation tensor scales with the base width; the per-interval layout holds
    // kSlices sequences of kIvLen bins per event instead of one of kBins
    size_t big = (size_t)kBigElems * (c0 / kC0), small = (size_t)kSmallElems * (c0 / kC0);
    if (c->per_interval) slot_elems(kIvLen, c0, kSlices, &big, &small);
    p.act_slot_big = align256((size_t)p.chunk * big * eb);
    p.act_slot_small = align256((size_t)p.chunk * small * eb);
    p.act = o; o += 5 * p.act_slot_big + 2 * p.act_slot_small;
    p.total = o + 256;
    return p;
}

}  // namespace

pvf_status pack_fc_from_blob(const void *blob, size_t bytes, float *out) {
    std::vector<HostLayer> layers;
    int c0 = 0;
    const pvf_status st = parse_blob(blob, bytes, 0, layers, &c0);
    if (st != PVF_OK) return st;
    std::vector<float> f32;
    const F32Layout L = f32_layout(c0);
    fill_f32(layers, L, c0, f32);
    std::memcpy(out, f32.data() + L.fc, sizeof(float) * kFcFloats);
    return PVF_OK;
}

}  // namespace pvf

using namespace pvf;

// Event pairs recorded around kernel launches while profiling is enabled.
struct Profiler {
    static constexpr int kPairs = 1024;
    bool on = false;
    std::vector<cudaEvent_t> ev;            // 2 * kPairs, created at enable
    std::vector<std::string> names;         // per recorded pair
    int used = 0;
    bool open = false;
};

static void prof_begin(void *ctx, const char *name, cudaStream_t s) {
    Profiler *p = static_cast<Profiler *>(ctx);
    p->open = false;
    if (!p->on || p->used >= Profiler::kPairs) return;
    if (cudaEventRecord(p->ev[2 * p->used], s) != cudaSuccess) return;
    p->names[p->used] = name;
    p->open = true;
}
static void prof_end(void *ctx, cudaStream_t s) {
    Profiler *p = static_cast<Profiler *>(ctx);
    if (!p->open) return;
    p->open = false;
    if (cudaEventRecord(p->ev[2 * p->used + 1], s) == cudaSuccess) ++p->used;
}

struct pvf_handle {
    Profiler prof;
    ProfHook hook;
    pvf_config cfg;
    Plan plan;
    unsigned char *pool;
    size_t front_smem;
    int c0;                                 // UNet base width
    F32Layout f32;
    ConvF32Weights cw;
    const float *fc, *enc1, *fin;
    UnetBuffers buf;
    TcNet tc;
    float act_scale[PVF_N_ACT_SCALES];
    pvf_schedule sched;                     // launch schedule (zeros: the defaults)
};

int pvf_handle_max_pv(const pvf_handle *h) { return h->cfg.max_pv_per_event; }
int pvf_handle_max_events(const pvf_handle *h) { return h->cfg.max_events; }
int pvf_handle_precision(const pvf_handle *h) { return h->cfg.precision; }

extern "C" {

int32_t pvf_version(void) { return (1 << 16) | 0; }

const char *pvf_status_str(pvf_status s) {
    switch (s) {
    case PVF_OK: return "ok";
    case PVF_ERR_INVALID_ARG: return "invalid argument";
    case PVF_ERR_POOL_TOO_SMALL: return "pool too small";
    case PVF_ERR_WEIGHTS: return "malformed or incompatible weight blob";
    case PVF_ERR_CUDA: return "CUDA runtime error";
    case PVF_ERR_TIMEOUT: return "bounded device wait timed out";
    case PVF_ERR_UNSUPPORTED: return "unsupported configuration";
    case PVF_WARN_EVENTS_SKIPPED: return "some events were bypassed";
    case PVF_WARN_TRUNCATED: return "some PV lists were truncated";
    }
    return "unknown status";
}

pvf_status pvf_pool_bytes_required(const pvf_config *cfg, size_t *out) {
    if (!out) return PVF_ERR_INVALID_ARG;
    pvf_status st = check_config(cfg);
    if (st != PVF_OK) return st;
    *out = make_plan(cfg).total;
    return PVF_OK;
}

pvf_status pvf_create(const void *blob, size_t blob_bytes, void *pool, size_t pool_bytes,
                      const pvf_config *cfg, pvf_stream_t stream_, pvf_handle **out) {
    if (!out) return PVF_ERR_INVALID_ARG;
    *out = nullptr;
    pvf_status st = check_config(cfg);
    if (st != PVF_OK) return st;
    if (!pool || reinterpret_cast<uintptr_t>(pool) % 256) return PVF_ERR_INVALID_ARG;
    std::vector<HostLayer> layers;
    st = parse_blob(blob, blob_bytes, cfg_c0(cfg), layers);
    if (st != PVF_OK) return st;
    const Plan plan = make_plan(cfg);
    if (pool_bytes < plan.total) return PVF_ERR_POOL_TOO_SMALL;
    if (cfg->precision == PVF_FP8_E4M3 && !cfg->fp8_act_scales) return PVF_ERR_UNSUPPORTED;
    if (cfg->precision != PVF_FP32 && !tc_supported(cfg->precision)) return PVF_ERR_UNSUPPORTED;

    pvf_handle *h = new (std::nothrow) pvf_handle();
    if (!h) return PVF_ERR_INVALID_ARG;
    h->cfg = *cfg;
    h->cfg.fp8_act_scales = nullptr;
    h->cfg.schedule = nullptr;
    h->sched = cfg->schedule ? *cfg->schedule : pvf_schedule{};
    for (int k = 0; k < 6; ++k) h->tc.ctas_per_sm[k] = h->sched.conv_ctas_per_sm[k];
    h->tc.iv = cfg->per_interval;
    h->plan = plan;
    h->pool = static_cast<unsigned char *>(pool);
    h->front_smem = front_smem_bytes(cfg->max_tracks_per_event, cfg->boundary_mm);
    h->c0 = cfg_c0(cfg);
    h->f32 = f32_layout(h->c0);
    h->cw.c0 = h->c0;
    for (int i = 0; i < PVF_N_ACT_SCALES; ++i)
        h->act_scale[i] = cfg->fp8_act_scales ? cfg->fp8_act_scales[i] : 1.0f;

    const float *w32 = reinterpret_cast<const float *>(h->pool + plan.f32w);
    h->fc = w32 + h->f32.fc;
    h->enc1 = w32 + h->f32.enc1;
    h->fin = w32 + h->f32.fin;
    for (int k = 0; k < 6; ++k) { h->cw.w[k] = w32 + h->f32.conv_w[k]; h->cw.b[k] = w32 + h->f32.conv_b[k]; }
    for (int k = 0; k < 3; ++k) { h->cw.uw[k] = w32 + h->f32.up_w[k]; h->cw.ub[k] = w32 + h->f32.up_b[k]; }
    unsigned char *act = h->pool + plan.act;
    h->buf.e1 = act;
    h->buf.e2 = act + plan.act_slot_big;
    h->buf.e3 = act + 2 * plan.act_slot_big;
    h->buf.deep = act + 3 * plan.act_slot_big;
    h->buf.up = act + 4 * plan.act_slot_big;
    h->buf.s0 = act + 5 * plan.act_slot_big;
    h->buf.s1 = act + 5 * plan.act_slot_big + plan.act_slot_small;
    h->buf.logits = reinterpret_cast<float *>(h->pool + plan.logits);
    h->tc.final_w = h->fin;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    std::vector<float> f32;
    fill_f32(layers, h->f32, h->c0, f32);
    std::vector<unsigned char> tcw;
    cudaError_t err = cudaSuccess;
    if (cfg->precision != PVF_FP32) {
        std::vector<LayerF32> views(kNumLayers);
        for (int i = 0; i < kNumLayers; ++i) {
            views[i].w = layers[i].w.data();
            views[i].b = layers[i].b.data();
            std::memcpy(views[i].shape, layers[i].shape, sizeof views[i].shape);
        }
        h->tc.status = reinterpret_cast<int32_t *>(h->pool + plan.status);
        // status word at 0, calibration maxima at 64, tile schedulers at 128 (zeroed below)
        h->tc.sched = reinterpret_cast<int32_t *>(h->pool + plan.status + 128);
        if (!tc_pack_weights(cfg->precision, views, h->act_scale, tcw, &h->tc, h->pool + plan.tcw)) {
            delete h;
            return PVF_ERR_WEIGHTS;
        }
    }
    if (err == cudaSuccess) err = cudaMemsetAsync(h->pool, 0, plan.f32w, s);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(h->pool + plan.f32w, f32.data(), f32.size() * sizeof(float),
                              cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess && !tcw.empty())
        err = cudaMemcpyAsync(h->pool + plan.tcw, tcw.data(), tcw.size(), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = cudaMemsetAsync(act, 0, plan.total - plan.act, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) {
        delete h;
        return PVF_ERR_CUDA;
    }
    *out = h;
    return PVF_OK;
}

pvf_status pvf_destroy(pvf_handle *h) {
    if (h) for (cudaEvent_t e : h->prof.ev) cudaEventDestroy(e);
    delete h;
    return PVF_OK;
}

pvf_status pvf_profile_enable(pvf_handle *h, int32_t on) {
    if (!h) return PVF_ERR_INVALID_ARG;
    if (on && h->prof.ev.empty()) {
        h->prof.ev.resize(2 * Profiler::kPairs);
        h->prof.names.resize(Profiler::kPairs);
        for (auto &e : h->prof.ev)
            if (cudaEventCreate(&e) != cudaSuccess) return PVF_ERR_CUDA;
    }
    h->prof.on = on != 0;
    h->prof.used = 0;
    h->hook.begin = prof_begin;
    h->hook.end = prof_end;
    h->hook.ctx = &h->prof;
    return PVF_OK;
}

pvf_status pvf_profile_read(pvf_handle *h, pvf_kernel_time *out, int32_t max_entries,
                            int32_t *n_entries, pvf_stream_t stream_) {
    if (!h || !n_entries || max_entries < 0 || (max_entries > 0 && !out)) return PVF_ERR_INVALID_ARG;
    *n_entries = 0;
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream_)) != cudaSuccess) return PVF_ERR_CUDA;
    std::vector<pvf_kernel_time> acc;
    for (int i = 0; i < h->prof.used; ++i) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, h->prof.ev[2 * i], h->prof.ev[2 * i + 1]) != cudaSuccess)
            return PVF_ERR_CUDA;
        const std::string &nm = h->prof.names[i];
        pvf_kernel_time *slot = nullptr;
        for (auto &k : acc) if (nm == k.name) slot = &k;
        if (!slot) {
            acc.push_back(pvf_kernel_time{});
            slot = &acc.back();
            std::strncpy(slot->name, nm.c_str(), sizeof slot->name - 1);
        }
        slot->launches += 1;
        slot->total_ms += ms;
    }
    h->prof.used = 0;
    const int n = (int)acc.size() < max_entries ? (int)acc.size() : max_entries;
    for (int i = 0; i < n; ++i) out[i] = acc[i];
    *n_entries = n;
    return PVF_OK;
}

static bool tracks_ok(const pvf_tracks_soa *t) {
    if (!t || t->n_tracks < 0) return false;
    for (int k = 0; k < PVF_N_FEATURES; ++k)
        if (!t->f[k] || reinterpret_cast<uintptr_t>(t->f[k]) % 4) return false;
    return true;
}

static bool aligned4(const void *p) { return reinterpret_cast<uintptr_t>(p) % 4 == 0; }
static bool aligned16(const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

// One chunk: front (steps 1-2 + enc1), UNet, tail (final conv + peaks).
// n_dyn (tensor-core forms, whole path only): device-side event count of the call, read
// by the front kernel and copied to a pool word for the kernels after it.
static cudaError_t run_chunk(pvf_handle *h, const pvf_tracks_soa *tracks, const int32_t *offsets,
                             const float *hist_in, const float *logit_in, int ev_base, int n,
                             float *pv_z, int32_t *pv_count, float *hist_out, float *logit_out,
                             bool run_front, bool run_unet, bool run_tail, cudaStream_t s,
                             const int32_t *n_dyn = nullptr, const int32_t *ev_index = nullptr) {
    int32_t *status = reinterpret_cast<int32_t *>(h->pool + h->plan.status);
    int32_t *flags = reinterpret_cast<int32_t *>(h->pool + h->plan.ev_flag);
    int32_t *n_copy = n_dyn ? reinterpret_cast<int32_t *>(h->pool + h->plan.status + kDynCountOff) : nullptr;
    const int prec = h->cfg.precision;
    cudaError_t err = cudaSuccess;
    const ProfHook *prof = h->prof.on ? &h->hook : nullptr;
    if (run_front) {
        ProfScope ps(prof, "front", s);
        FrontArgs a{};
        if (tracks) {
            for (int k = 0; k < kFeatures; ++k) a.feat[k] = tracks->f[k];
            a.n_tracks = tracks->n_tracks;
        }
        a.offsets = offsets;
        a.n_events = n;
        a.ev_base = ev_base;
        a.max_tracks = h->cfg.max_tracks_per_event;
        a.c0 = h->c0;
        a.iv = h->cfg.per_interval;
        a.edge = h->cfg.boundary_mm;
        a.edge_hi = 10.0f - h->cfg.boundary_mm;
        a.fc = h->fc;
        a.enc1 = h->enc1;
        a.hist_in = hist_in;
        a.hist_out = hist_out;
        a.e1 = h->buf.e1;
        a.p1 = h->buf.s0;
        a.e1_inv_scale = 1.0f / h->act_scale[kScaleL1];
        a.ev_flag = flags;
        a.status = status;
        a.amax = h->tc.amax;
        a.n_dyn = n_dyn;
        a.n_dyn_copy = n_copy;
        a.ev_index = ev_index;
        a.ctas_per_sm = h->sched.front_ctas_per_sm;
        if (prec == PVF_FP32) {
            err = launch_front(a, prec, h->front_smem, s);
        } else {
            a.fc_img = h->tc.fc_img;
            a.ev_ctr = reinterpret_cast<int32_t *>(h->pool + h->plan.status + kFrontCtrOff);
            err = launch_front_tc(a, prec, s);
        }
        if (err != cudaSuccess) return err;
    }
    if (run_unet) {
        if (prec == PVF_FP32) err = launch_unet_f32(h->cw, h->buf, n, h->cfg.per_interval != 0, s, prof);
        else err = launch_unet_tc(h->tc, h->buf, n, n_copy, ev_base, s, prof);
        if (err != cudaSuccess) return err;
    }
    if (run_tail) {
        ProfScope ps(prof, "tail", s);
        TailArgs t{};
        t.d1 = h->buf.deep;
        t.logit_in = logit_in;
        t.logit_in_base = 0;
        t.ev_flag = logit_in ? nullptr : flags;
        if (!logit_in && prec != PVF_FP32) {
            // tensor-core forms: the final conv ran in dec1's epilogue; peaks only
            t.logit_in = h->buf.logits;
            t.logit_in_base = ev_base;
        }
        t.d1_scale = h->act_scale[kScaleD1];
        t.final_w = h->fin;
        t.c0 = h->c0;
        t.iv = h->cfg.per_interval;
        t.n_events = n;
        t.ev_base = ev_base;
        t.logit_out = logit_out;
        t.pv_z = pv_z;
        t.pv_count = pv_count;
        t.max_pv = h->cfg.max_pv_per_event;
        t.status = status;
        t.n_dyn = n_copy;
        t.ctas_per_sm = h->sched.tail_ctas_per_sm;
        err = launch_tail(t, prec, s);
    }
    return err;
}

pvf_status pvf_infer_ex(pvf_handle *h, const pvf_tracks_soa *tracks, const int32_t *offsets,
                        int32_t n, float *pv_z, int32_t *pv_count, float *hist_out,
                        float *logit_out, pvf_stream_t stream_) {
    if (!h || n < 0 || n > h->cfg.max_events) return PVF_ERR_INVALID_ARG;
    if (n == 0) return PVF_OK;
    if (!tracks_ok(tracks) || !offsets || !aligned4(offsets) || !pv_z || !aligned4(pv_z) ||
        !pv_count || !aligned4(pv_count) || (hist_out && !aligned16(hist_out)) ||
        (logit_out && !aligned4(logit_out)))
        return PVF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    for (int c0 = 0; c0 < n; c0 += h->plan.chunk) {
        const int nc = n - c0 < h->plan.chunk ? n - c0 : h->plan.chunk;
        if (run_chunk(h, tracks, offsets, nullptr, nullptr, c0, nc, pv_z, pv_count, hist_out,
                      logit_out, true, true, true, s) != cudaSuccess)
            return PVF_ERR_CUDA;
    }
    return PVF_OK;
}

pvf_status pvf_infer(pvf_handle *h, const pvf_tracks_soa *tracks, const int32_t *offsets,
                     int32_t n, float *pv_z, int32_t *pv_count, pvf_stream_t stream) {
    return pvf_infer_ex(h, tracks, offsets, n, pv_z, pv_count, nullptr, nullptr, stream);
}

pvf_status pvf_stage_histogram(pvf_handle *h, const pvf_tracks_soa *tracks, const int32_t *offsets,
                               int32_t n, float *hist, pvf_stream_t stream_) {
    if (!h || n < 0 || n > h->cfg.max_events) return PVF_ERR_INVALID_ARG;
    if (n == 0) return PVF_OK;
    if (!tracks_ok(tracks) || !offsets || !aligned4(offsets) || !hist || !aligned16(hist))
        return PVF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    for (int c0 = 0; c0 < n; c0 += h->plan.chunk) {
        const int nc = n - c0 < h->plan.chunk ? n - c0 : h->plan.chunk;
        if (run_chunk(h, tracks, offsets, nullptr, nullptr, c0, nc, nullptr, nullptr, hist,
                      nullptr, true, false, false, s) != cudaSuccess)
            return PVF_ERR_CUDA;
    }
    return PVF_OK;
}

pvf_status pvf_stage_unet(pvf_handle *h, const float *hist, int32_t n, float *logit,
                          pvf_stream_t stream_) {
    if (!h || n < 0 || n > h->cfg.max_events) return PVF_ERR_INVALID_ARG;
    if (n == 0) return PVF_OK;
    if (!hist || !aligned4(hist) || !logit || !aligned4(logit)) return PVF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    for (int c0 = 0; c0 < n; c0 += h->plan.chunk) {
        const int nc = n - c0 < h->plan.chunk ? n - c0 : h->plan.chunk;
        if (run_chunk(h, nullptr, nullptr, hist, nullptr, c0, nc, nullptr, nullptr, nullptr, logit,
                      true, true, true, s) != cudaSuccess)
            return PVF_ERR_CUDA;
    }
    return PVF_OK;
}

pvf_status pvf_stage_peaks(pvf_handle *h, const float *logit, int32_t n, float *pv_z,
                           int32_t *pv_count, pvf_stream_t stream_) {
    if (!h || n < 0 || n > h->cfg.max_events) return PVF_ERR_INVALID_ARG;
    if (n == 0) return PVF_OK;
    if (!logit || !aligned4(logit) || !pv_z || !aligned4(pv_z) || !pv_count || !aligned4(pv_count))
        return PVF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    for (int c0 = 0; c0 < n; c0 += h->plan.chunk) {
        const int nc = n - c0 < h->plan.chunk ? n - c0 : h->plan.chunk;
        if (run_chunk(h, nullptr, nullptr, nullptr, logit, c0, nc, pv_z, pv_count, nullptr,
                      nullptr, false, false, true, s) != cudaSuccess)
            return PVF_ERR_CUDA;
    }
    return PVF_OK;
}

pvf_status pvf_calibrate(pvf_handle *h, const pvf_tracks_soa *tracks, const int32_t *offsets,
                         int32_t n, float *out_scales, pvf_stream_t stream_) {
    if (!h || n < 1 || n > h->cfg.max_events || !out_scales) return PVF_ERR_INVALID_ARG;
    if (h->cfg.precision != PVF_BF16) return PVF_ERR_UNSUPPORTED;
    if (!tracks_ok(tracks) || !offsets || !aligned4(offsets)) return PVF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    float *amax = reinterpret_cast<float *>(h->pool + h->plan.status + 64);
    if (cudaMemsetAsync(amax, 0, sizeof(float) * PVF_N_ACT_SCALES, s) != cudaSuccess) return PVF_ERR_CUDA;
    h->tc.amax = amax;
    cudaError_t err = cudaSuccess;
    for (int c0 = 0; c0 < n && err == cudaSuccess; c0 += h->plan.chunk) {
        const int nc = n - c0 < h->plan.chunk ? n - c0 : h->plan.chunk;
        err = run_chunk(h, tracks, offsets, nullptr, nullptr, c0, nc, nullptr, nullptr, nullptr,
                        nullptr, true, true, false, s);
    }
    h->tc.amax = nullptr;
    float host[PVF_N_ACT_SCALES];
    if (err != cudaSuccess ||
        cudaMemcpyAsync(host, amax, sizeof host, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PVF_ERR_CUDA;
    for (int i = 0; i < PVF_N_ACT_SCALES; ++i)
        out_scales[i] = (i < kNumScales && host[i] > 0.0f) ? host[i] / 448.0f : 1.0f;
    return PVF_OK;
}

}  // extern "C"

struct pvf_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

static pvf_status graph_create(pvf_handle *h, const pvf_tracks_soa *tracks, const int32_t *offsets,
                               const int32_t *n_dyn, int32_t n, float *pv_z, int32_t *pv_count,
                               pvf_graph **out, const int32_t *ev_index = nullptr) {
    if (!out) return PVF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!h || n < 1 || n > h->cfg.max_events) return PVF_ERR_INVALID_ARG;
    if (!tracks_ok(tracks) || !offsets || !aligned4(offsets) || !pv_z || !aligned4(pv_z) ||
        !pv_count || !aligned4(pv_count) || (n_dyn && !aligned4(n_dyn)))
        return PVF_ERR_INVALID_ARG;
    if ((n_dyn || ev_index) && h->cfg.precision == PVF_FP32) return PVF_ERR_UNSUPPORTED;
    if (ev_index && !aligned4(ev_index)) return PVF_ERR_INVALID_ARG;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return PVF_ERR_CUDA;
    const bool prof = h->prof.on;
    h->prof.on = false;
    pvf_graph *g = new (std::nothrow) pvf_graph();
    pvf_status st = g ? PVF_OK : PVF_ERR_INVALID_ARG;
    if (st == PVF_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        st = PVF_ERR_CUDA;
    if (st == PVF_OK) {
        cudaError_t err = cudaSuccess;
        for (int c0 = 0; c0 < n && err == cudaSuccess; c0 += h->plan.chunk) {
            const int nc = n - c0 < h->plan.chunk ? n - c0 : h->plan.chunk;
            err = run_chunk(h, tracks, offsets, nullptr, nullptr, c0, nc, pv_z, pv_count, nullptr,
                            nullptr, true, true, true, cs, n_dyn, ev_index);
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t end = cudaStreamEndCapture(cs, &graph);
        if (err != cudaSuccess || end != cudaSuccess || !graph) {
            st = PVF_ERR_CUDA;
            if (graph) cudaGraphDestroy(graph);
        } else {
            g->graph = graph;
            if (cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) st = PVF_ERR_CUDA;
        }
    }
    h->prof.on = prof;
    cudaStreamDestroy(cs);
    if (st != PVF_OK) {
        if (g) {
            if (g->exec) cudaGraphExecDestroy(g->exec);
            if (g->graph) cudaGraphDestroy(g->graph);
            delete g;
        }
        return st;
    }
    *out = g;
    return PVF_OK;
}

pvf_status pvf_graph_create(pvf_handle *h, const pvf_tracks_soa *tracks, const int32_t *offsets,
                            int32_t n, float *pv_z, int32_t *pv_count, pvf_graph **out) {
    return graph_create(h, tracks, offsets, nullptr, n, pv_z, pv_count, out);
}

pvf_status graph_create_gather(pvf_handle *h, const pvf_tracks_soa *store, const int32_t *store_offsets,
                               const int32_t *ev_index, const int32_t *n_events, int32_t max_n_events,
                               float *pv_z, int32_t *pv_count, pvf_graph **out) {
    if (!ev_index || !n_events) {
        if (out) *out = nullptr;
        return PVF_ERR_INVALID_ARG;
    }
    return graph_create(h, store, store_offsets, n_events, max_n_events, pv_z, pv_count, out, ev_index);
}

pvf_status pvf_graph_create_dynamic(pvf_handle *h, const pvf_tracks_soa *tracks, const int32_t *offsets,
                                    const int32_t *n_events, int32_t max_n_events, float *pv_z,
                                    int32_t *pv_count, pvf_graph **out) {
    if (!n_events) {
        if (out) *out = nullptr;
        return PVF_ERR_INVALID_ARG;
    }
    return graph_create(h, tracks, offsets, n_events, max_n_events, pv_z, pv_count, out);
}

pvf_status pvf_graph_launch(pvf_graph *g, pvf_stream_t stream) {
    if (!g || !g->exec) return PVF_ERR_INVALID_ARG;
    return cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? PVF_OK
                                                                                        : PVF_ERR_CUDA;
}

pvf_status pvf_graph_destroy(pvf_graph *g) {
    if (!g) return PVF_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return PVF_OK;
}

pvf_status pvf_test_wait_timeout(pvf_handle *h, int32_t n_events, uint32_t limit_us, pvf_stream_t stream_) {
    if (!h || n_events < 1 || n_events > h->cfg.max_events || n_events > h->plan.chunk || limit_us < 1 ||
        limit_us > 100000)
        return PVF_ERR_INVALID_ARG;
    if (h->cfg.precision == PVF_FP32) return PVF_ERR_UNSUPPORTED;
    return launch_stall_test_tc(h->tc, h->buf, n_events, limit_us, reinterpret_cast<cudaStream_t>(stream_)) ==
                   cudaSuccess
               ? PVF_OK
               : PVF_ERR_CUDA;
}

pvf_status pvf_last_device_status(pvf_handle *h, int32_t *out_status, pvf_stream_t stream_) {
    if (!h || !out_status) return PVF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    int32_t v = 0;
    int32_t *word = reinterpret_cast<int32_t *>(h->pool + h->plan.status);
    if (cudaMemcpyAsync(&v, word, sizeof v, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || cudaMemsetAsync(word, 0, sizeof v, s) != cudaSuccess)
        return PVF_ERR_CUDA;
    *out_status = v;
    return PVF_OK;
}

}  // extern "C"
