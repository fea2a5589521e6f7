/*
 * PVFinder FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may
 * load this library. It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (paper §2, "PVFinder Architecture for Real-Time Inference"): the
 * three-stage hybrid PVFinder inference for each collision event --
 *   1. a per-track fully connected network on nine track features, whose outputs are
 *      combined into a z-binned histogram of the 400 mm interaction region, divided
 *      into 40 intervals of 100 bins (4000 bins of 0.1 mm over [-100, 300) mm);
 *   2. a UNet-style 1D CNN turning the histogram into a per-bin PV probability;
 *   3. heuristic peak finding by local-maximum detection.
 * The paper does not print the layer shapes, activations, padding or peak-finder
 * constants; the readings used here (architecture 9-32-32-32-32-32-100 with
 * LeakyReLU(0.01) and softplus; UNet with 4 levels of c0/2c0/4c0/8c0 channels, c0 = 16
 * or 32, k5 zero "same" padding, maxpool 2, ConvTranspose k2 s2, skip concat
 * [upsampled, skip]; threshold 0.01, strict-left / non-strict-right local max over
 * +-5 bins, centroid over +-3 bins; slice-relative z as the third feature; optional
 * boundary tracks in a second interval and the per-interval UNet layout of §3) are
 * stated next to the code that uses them and listed in the design notes.
 *
 * Everything is a direct loop in double precision, in the order of the definition;
 * no blocking, fusion or reordering. Features arrive as float32 and are widened.
 * The slice index is the one integer decision taken in float32, because the slice
 * boundaries are defined on the float32 track z (see oracle_slice_index).
 *
 * Parity status: each stage is pinned by tests against closed forms, brute force or
 * library routines (see tests/test_oracle_pins.py). The end-to-end composition with
 * random He weights has no external pin beyond those stage pins and a second,
 * independently written numpy statement used in the tests.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_NBINS 4000
#define OR_NSLICES 40
#define OR_SLICE_BINS 100
#define OR_Z_LO (-100.0)
#define OR_BIN_W 0.1
#define OR_MAX_HIDDEN 64
#define OR_MAX_OUT 128

typedef struct {
    int c0;          /* UNet base width: levels have c0, 2c0, 4c0, 8c0 channels   */
    int fc_hidden;   /* FC hidden width (32)                                       */
    int fc_out;      /* FC output width = bins per slice (100)                     */
    const double *fc_w[6], *fc_b[6];   /* W[out][in], b[out]                        */
    const double *enc_w[4], *enc_b[4]; /* enc1..enc4: W[Cout][Cin][5]               */
    const double *up_w[3], *up_b[3];   /* up3, up2, up1: W[Cin][Cout][2]            */
    const double *dec_w[3], *dec_b[3]; /* dec3, dec2, dec1: W[Cout][2*Cout][5]      */
    const double *fin_w, *fin_b;       /* final: W[1][c0][5], b[1]                  */
} oracle_weights;

/* ------------------------------------------------------------------ elementary */

static double leaky(double x) { return x > 0.0 ? x : 0.01 * x; }

/* softplus(x) = log(1 + e^x); for x > 20 the correction log1p(e^-x) is below 2.1e-9
 * and x itself is returned. */
static double softplus(double x) { return x > 20.0 ? x : log1p(exp(x)); }

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* Slice (interval) index of a track, §2 "fixed spatial slicing ... 40 intervals of 100
 * bins". Slice s covers z in [-100 + 10 s, -90 + 10 s) mm. The division is taken in
 * float32 with round-to-nearest, floor((z + 100) / 10), so that a track exactly on a
 * boundary has one agreed slice. Returns -1 when the track is outside [0, 40) or z is
 * not finite. */
int oracle_slice_index(float z)
{
    volatile float t = z + 100.0f;
    volatile float q = t / 10.0f;
    if (!(q >= 0.0f && q < 40.0f)) return -1;
    return (int)floorf(q);
}

/* Per-track FC network, §2 ("six FC layers"): h1..h5 = LeakyReLU(W h + b), then
 * out = softplus(W6 h5 + b6). x[9] is the feature vector with feature 2 already
 * replaced by the slice-relative z. */
void oracle_fc_track(const oracle_weights *w, const double *x, double *out)
{
    const int H = w->fc_hidden, O = w->fc_out;
    double h[OR_MAX_HIDDEN], g[OR_MAX_HIDDEN];
    for (int o = 0; o < H; ++o) {
        double acc = w->fc_b[0][o];
        for (int i = 0; i < 9; ++i) acc += w->fc_w[0][o * 9 + i] * x[i];
        h[o] = leaky(acc);
    }
    for (int l = 1; l <= 4; ++l) {
        for (int o = 0; o < H; ++o) {
            double acc = w->fc_b[l][o];
            for (int i = 0; i < H; ++i) acc += w->fc_w[l][o * H + i] * h[i];
            g[o] = leaky(acc);
        }
        memcpy(h, g, sizeof(double) * (size_t)H);
    }
    for (int o = 0; o < O; ++o) {
        double acc = w->fc_b[5][o];
        for (int i = 0; i < H; ++i) acc += w->fc_w[5][o * H + i] * h[i];
        out[o] = softplus(acc);
    }
}

/* The second interval of a boundary track (§3: tracks on interval boundaries belong to
 * two intervals; the paper gives no width, so it is a parameter). A valid track of
 * slice s whose slice-relative position zr = z - (-100 + 10 s), taken in float32
 * round-to-nearest like the slice index, satisfies zr < edge belongs also to slice
 * s - 1 (if s > 0); one with zr >= 10 - edge (float32) also to slice s + 1 (if s < 39).
 * edge = 0 gives no second interval; 0 <= edge < 5, so a track has at most two.
 * Returns the second slice, or -1. */
int oracle_second_slice(float z, int s, float edge)
{
    if (s < 0 || !(edge > 0.0f)) return -1;
    volatile float base = -100.0f + 10.0f * (float)s;
    volatile float zr = z - base;
    volatile float hi = 10.0f - edge;
    if (s > 0 && zr < edge) return s - 1;
    if (s < OR_NSLICES - 1 && zr >= hi) return s + 1;
    return -1;
}

/* Histogram of one event (§2: "combining each track's contribution"): every valid track
 * adds its fc_out outputs to the bins of its own slice and, if it is a boundary track
 * (oracle_second_slice), the outputs of a second evaluation to the bins of its second
 * slice; tracks are summed in input order. A track is dropped when any feature is not
 * finite or its slice is outside [0, 40). Feature 2 fed to the net is z - (-100 + 10 s),
 * the position relative to the start of the slice s being filled, in mm (in a second
 * slice it lies just outside [0, 10)). Returns the number of dropped tracks. */
int oracle_event_histogram(const float *const feats[9], int64_t begin, int64_t end,
                           const oracle_weights *w, float edge, double *hist /* [4000] */)
{
    double x[9], out[OR_MAX_OUT];
    int dropped = 0;
    memset(hist, 0, sizeof(double) * OR_NBINS);
    for (int64_t t = begin; t < end; ++t) {
        int finite = 1;
        for (int k = 0; k < 9; ++k) {
            x[k] = (double)feats[k][t];
            if (!isfinite(x[k])) finite = 0;
        }
        int s = finite ? oracle_slice_index(feats[2][t]) : -1;
        if (s < 0) { ++dropped; continue; }
        const double z = x[2];
        x[2] = z - (OR_Z_LO + 10.0 * (double)s);
        oracle_fc_track(w, x, out);
        for (int j = 0; j < w->fc_out; ++j) hist[s * OR_SLICE_BINS + j] += out[j];
        const int s2 = oracle_second_slice(feats[2][t], s, edge);
        if (s2 >= 0) {
            x[2] = z - (OR_Z_LO + 10.0 * (double)s2);
            oracle_fc_track(w, x, out);
            for (int j = 0; j < w->fc_out; ++j) hist[s2 * OR_SLICE_BINS + j] += out[j];
        }
    }
    return dropped;
}

/* ------------------------------------------------------------------ UNet pieces */

/* Conv1d, kernel 5, zero padding 2, channel-major [C][L]:
 * y[co][i] = b[co] + sum_ci sum_t W[co][ci][t] * x[ci][i + t - 2]. No activation. */
void oracle_conv1d_k5(const double *x, int cin, int L, const double *W, const double *b,
                      int cout, double *y)
{
    for (int co = 0; co < cout; ++co)
        for (int i = 0; i < L; ++i) {
            double acc = b[co];
            for (int ci = 0; ci < cin; ++ci)
                for (int t = 0; t < 5; ++t) {
                    int j = i + t - 2;
                    if (j < 0 || j >= L) continue;
                    acc += W[((size_t)co * cin + ci) * 5 + t] * x[(size_t)ci * L + j];
                }
            y[(size_t)co * L + i] = acc;
        }
}

/* ConvTranspose1d, kernel 2, stride 2 (no overlap): input [Cin][L] -> output [Cout][2L],
 * y[co][2i + r] = b[co] + sum_ci W[ci][co][r] * x[ci][i]. No activation. */
void oracle_convT_k2s2(const double *x, int cin, int L, const double *W, const double *b,
                       int cout, double *y)
{
    for (int co = 0; co < cout; ++co)
        for (int i = 0; i < L; ++i)
            for (int r = 0; r < 2; ++r) {
                double acc = b[co];
                for (int ci = 0; ci < cin; ++ci)
                    acc += W[((size_t)ci * cout + co) * 2 + r] * x[(size_t)ci * L + i];
                y[(size_t)co * 2 * L + 2 * i + r] = acc;
            }
}

/* MaxPool1d(2, stride 2): [C][L] -> [C][L/2]. */
void oracle_maxpool2(const double *x, int C, int L, double *y)
{
    for (int c = 0; c < C; ++c)
        for (int i = 0; i < L / 2; ++i) {
            double a = x[(size_t)c * L + 2 * i], bb = x[(size_t)c * L + 2 * i + 1];
            y[(size_t)c * (L / 2) + i] = a > bb ? a : bb;
        }
}

static void leaky_inplace(double *x, size_t n) { for (size_t i = 0; i < n; ++i) x[i] = leaky(x[i]); }

/* Channel concat [a (first), b (second)] of two [C][L] tensors. */
static void concat2(const double *a, int ca, const double *b, int cb, int L, double *y)
{
    memcpy(y, a, sizeof(double) * (size_t)ca * L);
    memcpy(y + (size_t)ca * L, b, sizeof(double) * (size_t)cb * L);
}

/* Indices of the optional activation dumps of oracle_unet. */
enum { ACT_E1, ACT_P1, ACT_E2, ACT_P2, ACT_E3, ACT_P3, ACT_E4, ACT_U3, ACT_D3, ACT_U2,
       ACT_D2, ACT_U1, ACT_D1, ACT_F, ACT_PROB, ACT_N };

/* UNet-style 1D CNN of §2 on one event's histogram [1][L] (L divisible by 8):
 *   encoder  e1 = lrelu(conv(h)),  p1 = pool(e1)        c0  @ L
 *            e2 = lrelu(conv(p1)), p2 = pool(e2)        2c0 @ L/2
 *            e3 = lrelu(conv(p2)), p3 = pool(e3)        4c0 @ L/4
 *            e4 = lrelu(conv(p3))                        8c0 @ L/8
 *   decoder  u3 = lrelu(convT(e4)); d3 = lrelu(conv([u3, e3]))   4c0 @ L/4
 *            u2 = lrelu(convT(d3)); d2 = lrelu(conv([u2, e2]))   2c0 @ L/2
 *            u1 = lrelu(convT(d2)); d1 = lrelu(conv([u1, e1]))   c0  @ L
 *   head     f = conv(d1) (the logit), prob = sigmoid(f)        1   @ L
 * logit and prob are [L] outputs (either may be NULL); acts (nullable) receives copies of
 * the intermediates, indexed by the ACT_* enum. */
int oracle_unet(const oracle_weights *w, const double *hist, int L, double *logit,
                double *prob, double *const *acts)
{
    if (L <= 0 || L % 8) return -1;
    const int c1 = w->c0, c2 = 2 * c1, c3 = 4 * c1, c4 = 8 * c1;
    const int L1 = L, L2 = L / 2, L3 = L / 4, L4 = L / 8;
    size_t n_e1 = (size_t)c1 * L1, n_e2 = (size_t)c2 * L2, n_e3 = (size_t)c3 * L3,
           n_e4 = (size_t)c4 * L4;
    double *e1 = malloc(sizeof(double) * n_e1), *p1 = malloc(sizeof(double) * n_e1 / 2);
    double *e2 = malloc(sizeof(double) * n_e2), *p2 = malloc(sizeof(double) * n_e2 / 2);
    double *e3 = malloc(sizeof(double) * n_e3), *p3 = malloc(sizeof(double) * n_e3 / 2);
    double *e4 = malloc(sizeof(double) * n_e4);
    double *u3 = malloc(sizeof(double) * n_e3), *d3 = malloc(sizeof(double) * n_e3);
    double *u2 = malloc(sizeof(double) * n_e2), *d2 = malloc(sizeof(double) * n_e2);
    double *u1 = malloc(sizeof(double) * n_e1), *d1 = malloc(sizeof(double) * n_e1);
    double *cat = malloc(sizeof(double) * 2 * n_e1);
    double *f = malloc(sizeof(double) * (size_t)L1);
    int rc = 0;
    if (!e1 || !p1 || !e2 || !p2 || !e3 || !p3 || !e4 || !u3 || !d3 || !u2 || !d2 || !u1 ||
        !d1 || !cat || !f) { rc = -2; goto done; }

    oracle_conv1d_k5(hist, 1, L1, w->enc_w[0], w->enc_b[0], c1, e1); leaky_inplace(e1, n_e1);
    oracle_maxpool2(e1, c1, L1, p1);
    oracle_conv1d_k5(p1, c1, L2, w->enc_w[1], w->enc_b[1], c2, e2); leaky_inplace(e2, n_e2);
    oracle_maxpool2(e2, c2, L2, p2);
    oracle_conv1d_k5(p2, c2, L3, w->enc_w[2], w->enc_b[2], c3, e3); leaky_inplace(e3, n_e3);
    oracle_maxpool2(e3, c3, L3, p3);
    oracle_conv1d_k5(p3, c3, L4, w->enc_w[3], w->enc_b[3], c4, e4); leaky_inplace(e4, n_e4);

    oracle_convT_k2s2(e4, c4, L4, w->up_w[0], w->up_b[0], c3, u3); leaky_inplace(u3, n_e3);
    concat2(u3, c3, e3, c3, L3, cat);
    oracle_conv1d_k5(cat, 2 * c3, L3, w->dec_w[0], w->dec_b[0], c3, d3); leaky_inplace(d3, n_e3);

    oracle_convT_k2s2(d3, c3, L3, w->up_w[1], w->up_b[1], c2, u2); leaky_inplace(u2, n_e2);
    concat2(u2, c2, e2, c2, L2, cat);
    oracle_conv1d_k5(cat, 2 * c2, L2, w->dec_w[1], w->dec_b[1], c2, d2); leaky_inplace(d2, n_e2);

    oracle_convT_k2s2(d2, c2, L2, w->up_w[2], w->up_b[2], c1, u1); leaky_inplace(u1, n_e1);
    concat2(u1, c1, e1, c1, L1, cat);
    oracle_conv1d_k5(cat, 2 * c1, L1, w->dec_w[2], w->dec_b[2], c1, d1); leaky_inplace(d1, n_e1);

    oracle_conv1d_k5(d1, c1, L1, w->fin_w, w->fin_b, 1, f);
    for (int i = 0; i < L1; ++i) {
        if (logit) logit[i] = f[i];
        if (prob) prob[i] = sigmoid(f[i]);
    }

    if (acts) {
        for (int i = 0; i < L1; ++i) cat[i] = sigmoid(f[i]);
        const double *src[ACT_N] = {e1, p1, e2, p2, e3, p3, e4, u3, d3, u2, d2, u1, d1, f, cat};
        const size_t cnt[ACT_N] = {n_e1, n_e1 / 2, n_e2, n_e2 / 2, n_e3, n_e3 / 2, n_e4, n_e3,
                                   n_e3, n_e2, n_e2, n_e1, n_e1, (size_t)L1, (size_t)L1};
        for (int k = 0; k < ACT_N; ++k)
            if (acts[k]) memcpy(acts[k], src[k], sizeof(double) * cnt[k]);
    }
done:
    free(e1); free(p1); free(e2); free(p2); free(e3); free(p3); free(e4);
    free(u3); free(d3); free(u2); free(d2); free(u1); free(d1); free(cat); free(f);
    return rc;
}

/* ------------------------------------------------------------------ peak finding */

/* Peak finding of §2 ("heuristic peak finding", "local maximum detection") with a fixed
 * threshold in place of the paper's learned thresholds. The decisions are defined on the
 * probabilities p = sigmoid(f); because sigmoid is strictly increasing they are taken,
 * exactly, on the logits f:  p[i] > p[j] <=> f[i] > f[j]  and  p[i] > thr <=>
 * f[i] > thr_logit = ln(thr / (1 - thr)). (Comparing p after rounding would replace the
 * decision by a rounding artefact wherever sigmoid saturates: double rounds it to 1 for
 * f > 36.7.) Bin i is a PV candidate iff
 *   f[i] > thr_logit,  f[i] > f[j] for j in [i-hw, i-1],  f[i] >= f[j] for j in [i+1, i+hw],
 * windows clipped to [0, L-1] (the leftmost bin of a plateau wins). Its z is the centroid
 * over [i-hc, i+hc] clipped: sum p[j] zc(j) / sum p[j], zc(j) = z_lo + (j + 0.5) bw, with
 * the probabilities p as weights. PVs come out in ascending z. Returns the true count;
 * writes at most max_pv. */
int oracle_peaks(const double *f, const double *p, int L, double thr_logit, int hw, int hc,
                 double z_lo, double bw, int max_pv, double *z_out, int32_t *bin_out)
{
    int n = 0;
    for (int i = 0; i < L; ++i) {
        if (!(f[i] > thr_logit)) continue;
        int is_max = 1;
        for (int j = i - hw; j < i && is_max; ++j)
            if (j >= 0 && !(f[i] > f[j])) is_max = 0;
        for (int j = i + 1; j <= i + hw && is_max; ++j)
            if (j < L && !(f[i] >= f[j])) is_max = 0;
        if (!is_max) continue;
        if (n < max_pv) {
            double num = 0.0, den = 0.0;
            for (int j = i - hc; j <= i + hc; ++j) {
                if (j < 0 || j >= L) continue;
                num += p[j] * (z_lo + ((double)j + 0.5) * bw);
                den += p[j];
            }
            if (z_out) z_out[n] = num / den;
            if (bin_out) bin_out[n] = i;
        }
        ++n;
    }
    return n;
}

/* Per-interval layout (§3: the CNN input has a batch dimension of 40 spatial intervals):
 * each interval runs the UNet as its own sequence of OR_IV_LEN bins -- its 100 bins with
 * OR_IV_PAD zero bins on each side, the fewest that survive three 2:1 poolings -- and its
 * 100 central logits become bins [100 s, 100 s + 100) of the event's logits. prob (may be
 * NULL) receives sigmoid of the assembled logits. Returns 0, or -2 when out of memory. */
#define OR_IV_PAD 2
#define OR_IV_LEN (OR_SLICE_BINS + 2 * OR_IV_PAD)
int oracle_unet_intervals(const oracle_weights *w, const double *hist, double *logit, double *prob)
{
    double xw[OR_IV_LEN], fw[OR_IV_LEN];
    for (int s = 0; s < OR_NSLICES; ++s) {
        for (int j = 0; j < OR_IV_LEN; ++j) {
            const int b = j - OR_IV_PAD;
            xw[j] = (b >= 0 && b < OR_SLICE_BINS) ? hist[s * OR_SLICE_BINS + b] : 0.0;
        }
        if (oracle_unet(w, xw, OR_IV_LEN, fw, NULL, NULL) != 0) return -2;
        for (int b = 0; b < OR_SLICE_BINS; ++b) logit[s * OR_SLICE_BINS + b] = fw[OR_IV_PAD + b];
    }
    if (prob)
        for (int i = 0; i < OR_NBINS; ++i) prob[i] = sigmoid(logit[i]);
    return 0;
}

/* ------------------------------------------------------------------ whole event */

typedef struct {
    const float *const *feats;
    const int32_t *offsets;
    int64_t n_tracks_total;
    int n_events;
    int max_tracks_per_event;
    const oracle_weights *w;
    double *hist_out, *logit_out, *prob_out;   /* nullable, [n_events][4000] */
    double *pv_z;                  /* [n_events][max_pv] */
    int32_t *pv_count;             /* [n_events] */
    int32_t *n_dropped;            /* nullable, [n_events] */
    int max_pv;
    double thr;
    float edge;
    int per_interval;
    int tid, nthreads;
    int rc;
} infer_job;

/* An event is processed iff 0 <= off[e] <= off[e+1] <= n_tracks_total and it holds at
 * most max_tracks_per_event tracks; otherwise it is bypassed (§3: events failing
 * validation bypass ML reconstruction) with pv_count = -1, and its z slots, hist,
 * logit and prob rows are left untouched. */
static void *infer_worker(void *arg)
{
    infer_job *j = (infer_job *)arg;
    double *hist = malloc(sizeof(double) * OR_NBINS);
    double *logit = malloc(sizeof(double) * OR_NBINS);
    double *prob = malloc(sizeof(double) * OR_NBINS);
    const double thr_logit = log(j->thr / (1.0 - j->thr));
    if (!hist || !logit || !prob) { j->rc = -2; free(hist); free(logit); free(prob); return NULL; }
    for (int e = j->tid; e < j->n_events; e += j->nthreads) {
        int64_t a = j->offsets[e], b = j->offsets[e + 1];
        if (a < 0 || b < a || b > j->n_tracks_total || (b - a) > j->max_tracks_per_event) {
            j->pv_count[e] = -1;
            continue;
        }
        int drop = oracle_event_histogram(j->feats, a, b, j->w, j->edge, hist);
        if (j->n_dropped) j->n_dropped[e] = drop;
        const int rc = j->per_interval ? oracle_unet_intervals(j->w, hist, logit, prob)
                                       : oracle_unet(j->w, hist, OR_NBINS, logit, prob, NULL);
        if (rc != 0) { j->rc = -2; break; }
        j->pv_count[e] = oracle_peaks(logit, prob, OR_NBINS, thr_logit, 5, 3, OR_Z_LO, OR_BIN_W,
                                      j->max_pv, j->pv_z + (size_t)e * j->max_pv, NULL);
        if (j->hist_out) memcpy(j->hist_out + (size_t)e * OR_NBINS, hist, sizeof(double) * OR_NBINS);
        if (j->logit_out) memcpy(j->logit_out + (size_t)e * OR_NBINS, logit, sizeof(double) * OR_NBINS);
        if (j->prob_out) memcpy(j->prob_out + (size_t)e * OR_NBINS, prob, sizeof(double) * OR_NBINS);
    }
    free(hist); free(logit); free(prob);
    return NULL;
}

/* Full inference over a batch of events, statically round-robin over nthreads threads
 * (nthreads <= 1 runs on the calling thread); edge is the boundary-track width in mm
 * (oracle_second_slice, 0 = none); per_interval selects the per-interval UNet layout
 * (oracle_unet_intervals). Returns 0 on success. */
int oracle_infer(const float *const feats[9], const int32_t *offsets, int64_t n_tracks_total,
                 int n_events, int max_tracks_per_event, const oracle_weights *w,
                 double *hist_out, double *logit_out, double *prob_out, double *pv_z,
                 int32_t *pv_count,
                 int32_t *n_dropped, int max_pv, double thr, float edge, int per_interval,
                 int nthreads)
{
    if (n_events < 0 || max_pv < 0 || !w || (n_events > 0 && (!offsets || !pv_z || !pv_count)))
        return -1;
    if (!(edge >= 0.0f && edge < 5.0f)) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n_events) nthreads = n_events > 0 ? n_events : 1;
    infer_job *jobs = calloc((size_t)nthreads, sizeof(infer_job));
    pthread_t *th = calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -2; }
    for (int t = 0; t < nthreads; ++t) {
        infer_job *j = &jobs[t];
        j->feats = feats; j->offsets = offsets; j->n_tracks_total = n_tracks_total;
        j->n_events = n_events; j->max_tracks_per_event = max_tracks_per_event; j->w = w;
        j->hist_out = hist_out; j->logit_out = logit_out; j->prob_out = prob_out; j->pv_z = pv_z; j->pv_count = pv_count;
        j->n_dropped = n_dropped; j->max_pv = max_pv; j->thr = thr; j->edge = edge;
        j->per_interval = per_interval; j->tid = t;
        j->nthreads = nthreads; j->rc = 0;
    }
    int rc = 0;
    if (nthreads == 1) {
        infer_worker(&jobs[0]);
    } else {
        int started = 0;
        for (int t = 0; t < nthreads; ++t) {
            if (pthread_create(&th[t], NULL, infer_worker, &jobs[t]) != 0) { rc = -3; break; }
            ++started;
        }
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    }
    for (int t = 0; t < nthreads; ++t) if (jobs[t].rc) rc = jobs[t].rc;
    free(jobs); free(th);
    return rc;
}
