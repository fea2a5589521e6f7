// Step 3 of the path (§2, UNet-style 1D CNN) on the fifth-generation tensor cores:
// every k5 convolution is an implicit GEMM over channels, M = 128 positions of one
// event, N = C_out, K = 5 taps x C_in, issued as tcgen05.mma with the accumulator in
// TMEM. The paper projects the gain of tensor cores and reduced precision (§5, Table 2);
// here they are the BF16, FP16 and FP8 (E4M3) forms.
//
// Kernel families (each a persistent, warp-specialised kernel):
//   enc2      conv 16->32  @2000, epilogue also writes the 2:1 max-pool
//   enc3      conv 32->64  @1000, + pool
//   enc4_up3  conv 64->128 @500,  epilogue feeds a second GEMM: ConvT 128->64 (k2 s2)
//   dec3_up2  conv [64|64]->64 @1000, + ConvT 64->32
//   dec2_up1  conv [32|32]->32 @2000, + ConvT 32->16
//   dec1      conv [16|16]->16 @4000, + the final conv 16->1 (logits)
// The skip concat is never materialised: the two inputs are copied into adjacent
// K-planes of the same shared-memory tile. Every conv and ConvT output goes through
// LeakyReLU(0.01) in the epilogue; the fused ConvT reads the conv tile from shared
// memory, so the deepest level's activations (e4, d3, d2) never reach global memory.
//
// Warp roles: warp 0 issues the bulk copies (weights once, then one halo'd activation
// tile per 128 positions into a ring of stages); warp 1 allocates TMEM and one thread
// issues the MMAs into NB accumulator buffers, so the MMAs of tile i wait only for the
// epilogue of tile i - NB; the remaining one, two or four warpgroups are the epilogue,
// one TMEM lane (= output position) per thread. With a fused ConvT and two or four
// epilogue warpgroups they split by role: half of them turn each conv accumulator into
// the ConvT's shared-memory operand, the other half store the ConvT output (written over
// the conv columns, already read) and free the buffer, so the operand of tile i is ready
// while the tensor core still runs the conv of tile i + 1; the two warpgroups of a role
// (if four) split its columns. Otherwise two warpgroups split the accumulator columns.
//
// Tap pairing (the 16-bit forms' dec3_up2 and dec2_up1): a tcgen05.mma costs about the same for
// N up to 64 (reading A dominates), so the small-C_out convs stack two taps' weights in N:
// per K step, taps (0, 1) on the tile as is, taps (2, 3) on the tile two rows down and tap
// 4 four rows down, accumulating E (taps 0, 2, 4 of row r) and O (taps 1, 3 of row r - 1)
// side by side. The conv at row r is E[r] + O[r + 1]: a one-lane shuffle, and through
// shared memory across the warps' lane quarters. Row 127 of a tile lacks O[128], so
// paired tiles advance by 127 rows. Three MMAs per K step replace five.
//
// Tiles: a CTA takes tiles blockIdx.x, + gridDim.x, ... In the many-CTA encoder kernels
// (DYN) the producer instead takes the next index from a global counter and hands it to
// the MMA thread and the epilogue through a small ring in shared memory (its own
// mbarriers), so CTAs that progress faster take more tiles: with a static stride the six
// CTAs sharing an SM finished their equal shares up to 50% apart. The last CTA to finish
// resets the counter for the next launch. In the other kernels the ring's handshake per
// tile measured slower than the imbalance it removes.
//
// Launch: programmatic dependent launch. The prologue (weights, parameters, barriers,
// TMEM) runs before griddepcontrol.wait, i.e. while the previous kernel finishes; the
// kernel then lets the next one launch. Every wait is bounded (1 s); on timeout the
// kernel records PVF_ERR_TIMEOUT, drains its own copies and MMAs, frees TMEM and returns.
#include "pvf_tc.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace pvf {
namespace {

using namespace tc;

constexpr int kTileM = 128;

// EPI_CONVT: the kernel's GEMM is itself a ConvT k2 s2 (one "tap", N = r * CUP + co), for
// the wide network's layers whose conv is split over CTAs and so cannot fuse its ConvT.
enum { EPI_STORE = 0, EPI_POOL = 1, EPI_UP = 2, EPI_FINAL = 3, EPI_CONVT = 4 };

__host__ __device__ constexpr int pow2ceil(int x) {
    int p = 32;
    while (p < x) p <<= 1;
    return p;
}
__host__ __device__ constexpr int align_up(int x, int a) { return (x + a - 1) / a * a; }

template <int PREC_, int CA_, int CB_, int COUT_, int L_, int EPI_, int CUP_, int STAGES_, int EWG_ = 1,
          int MAXREG_ = 128, int NB_ = 2, bool PAIRED_ = false, bool DYN_ = false, bool A2T_ = false,
          int SEQ_ = 0, int NSPLIT_ = 1>
struct Cfg {
    static constexpr int PREC = PREC_;
    static constexpr int ES = is16(PREC) ? 2 : 1;            // bytes per element
    static constexpr int PW = 16 / ES;                       // channels per 16-byte plane row
    static constexpr int CA = CA_, CB = CB_, CIN = CA_ + CB_, COUT = COUT_, L = L_, EPI = EPI_;
    static constexpr int CUP = CUP_;
    static constexpr int STAGES = STAGES_;
    static constexpr int EWG = EWG_;                         // epilogue warpgroups
    static constexpr int THREADS = 64 + 128 * EWG;
    // register cap: a warp's registers come from one SM sub-partition's 16K, so k CTAs of
    // 6 warps fit when 6k/4 (rounded up) warps x regs x 32 <= 16384
    static constexpr int MAXREG = MAXREG_;
    // TMEM accumulator buffers: the MMAs of tile i wait only for the epilogue of tile i - NB
    static constexpr int NB = NB_;
    static constexpr int EPI_COLS = COUT / EWG;              // conv columns per epilogue thread
    // columns per TMEM load of the conv epilogue for nc columns, and (paired taps) the
    // exchanges on xready per tile: one per load
    static constexpr int ldw(int nc) { return nc % 32 == 0 && (EWG == 2 || EPI == EPI_UP) ? 32 : 16; }
    static constexpr int xchunks(int nc) { return nc / ldw(nc); }
    static constexpr int PA = CA / PW, PB = CB / PW, PIN = PA + PB, POUT = COUT / PW;
    // A single input plane is half an MMA's K (32 bytes): pair taps (2j, 2j+1) in one MMA
    // by pointing the K-adjacent core matrix at the next row; a 6th zero tap pads.
    static constexpr bool PAIR = PIN == 1;
    static constexpr int TAPS = EPI == EPI_CONVT ? 1 : PAIR ? 6 : 5;
    static constexpr int ROWS = kTileM + TAPS - 1;           // halo'd tile rows
    // the tile's first storage row relative to its first position: 0 for the k5 convs (the
    // halo starts two rows before), kPad for the ConvT GEMM (row p + 2 holds position p)
    static constexpr int ROW_OFF = EPI == EPI_CONVT ? kPad : 0;
    // the layer's N split over NSPLIT groups of CTAs (CTA b computes part b % NSPLIT: COUT
    // of the NSPLIT * COUT output channels, or of the N columns of a ConvT GEMM), for the
    // wide network's layers whose whole weight image exceeds shared memory
    static constexpr int NSPLIT = NSPLIT_;
    static constexpr int POUT_TOT = NSPLIT * (COUT_ / (16 / (is16(PREC_) ? 2 : 1)));
    static constexpr int ROWS_E = L + 2 * kPad;              // storage rows per event
    static constexpr bool PAIRED = PAIRED_;                 // taps stacked in pairs along N
    // per-interval layout: the event is kSlices sequences laid end to end, SEQ storage rows
    // each (two zero rows, then its LSEQ positions), and two more zero rows after the last;
    // neighbouring sequences share the two zero rows between them (the k5 conv's padding on
    // either side), so the event's L = kSlices SEQ - 2 positions include those rows;
    // 0: one sequence of L
    static constexpr int SEQ = SEQ_;
    static constexpr int LSEQ = SEQ ? SEQ - kPad : L_;
    static constexpr int SEQP = SEQ ? LSEQ / 2 + kPad : 0;   // after the 2:1 pool
    static constexpr int SEQU = SEQ ? 2 * LSEQ + kPad : 0;   // after the ConvT
    static constexpr int64_t ROWS_P = SEQ ? (int64_t)kSlices * SEQP + kPad : L_ / 2 + 2 * kPad;  // pooled rows per event
    static constexpr int64_t ROWS_O = SEQ ? (int64_t)kSlices * SEQU + kPad : 2 * L_ + 2 * kPad;  // ConvT rows per event
    static constexpr bool DYN = DYN_;                       // tiles from the global counter
    // output rows per tile: row 127 of a paired tile lacks O[128]; the fused final conv
    // also needs two rows on each side
    static constexpr int ROWS_OK = PAIRED ? kTileM - 1 : kTileM;
    static constexpr int STRIDE = EPI == EPI_FINAL ? ROWS_OK - 2 * kPad : ROWS_OK;
    static constexpr int TPE = (L + STRIDE - 1) / STRIDE;    // tiles per event
    static constexpr int A_STAGE = align_up(PIN * ROWS * 16, 128);
    static constexpr int W_BYTES = TAPS * PIN * COUT * 16;
    static constexpr int N2 = EPI == EPI_UP ? 2 * CUP : 0;   // fused ConvT: n = r * CUP + co
    static constexpr int P2 = COUT / PW;                     // K-planes of the fused GEMM
    static constexpr int W2_BYTES = EPI == EPI_UP ? P2 * N2 * 16 : 0;
    // the fused ConvT's A operand (the conv output of the tile, quantised): in shared memory,
    // or (A2T) in tensor memory, written by the epilogue with tcgen05.st and read by the
    // MMA directly, which takes its traffic off the shared-memory pipe
    static constexpr bool A2T = A2T_ && EPI == EPI_UP;
    static constexpr int A2_BYTES = EPI == EPI_UP && !A2T ? P2 * kTileM * 16 : 0;
    static constexpr int A2_COLS = A2T ? P2 * 4 : 0;         // a 16-byte plane row = 4 columns
    // accumulator buffer: the fused ConvT writes its result over the conv columns, which
    // the epilogue has read before the ConvT's operand is complete
    static constexpr int CONV_COLS = PAIRED ? 2 * COUT : COUT;      // E | O when paired
    static constexpr int COLS_BUF = CONV_COLS > N2 ? CONV_COLS : N2;
    static constexpr int UP_OFF = 0;
    static constexpr int A2_COL0 = NB * COLS_BUF;            // A2 buffers after the accumulators
    static constexpr int TMEM_COLS = pow2ceil(NB * COLS_BUF + 2 * A2_COLS);
    // float parameters kept in shared memory: bias, bias2, column scales, final conv
    static constexpr int NPAR = 2 * (COUT + N2) + (EPI == EPI_FINAL ? 5 * COUT + 1 : 0);
    static constexpr int OFF_W = 0;
    static constexpr int OFF_W2 = align_up(OFF_W + W_BYTES, 128);
    static constexpr int OFF_PAR = align_up(OFF_W2 + W2_BYTES, 128);
    static constexpr int OFF_A = align_up(OFF_PAR + 4 * NPAR, 128);
    static constexpr int OFF_A2 = OFF_A + STAGES * A_STAGE;
    static constexpr int OFF_G = align_up(OFF_A2 + 2 * A2_BYTES, 128);
    static constexpr int G_BYTES = EPI == EPI_FINAL ? 2 * 5 * kTileM * 4 : 0;
    // paired: each lane quarter's first O row, for the quarter above (two buffers)
    static constexpr int OFF_X = align_up(OFF_G + G_BYTES, 128);
    static constexpr int X_BYTES = PAIRED ? 2 * 4 * COUT * 4 : 0;
    static constexpr int OFF_BAR = align_up(OFF_X + X_BYTES, 128);
    static constexpr int SMEM = OFF_BAR + 512;
    // instruction-descriptor operand format: kind::f16 0 = f16, 1 = bf16; kind::f8f6f4 0 = e4m3
    static constexpr uint32_t FMT = PREC == PVF_BF16 ? 1u : 0u;
    static constexpr uint32_t IDESC1 = idesc_f32acc(kTileM, COUT, FMT);
    static constexpr uint32_t IDESC2 = idesc_f32acc(kTileM, N2 > 0 ? N2 : 16, FMT);
    static_assert(COUT % 16 == 0 && COUT <= 256, "MMA N");
    static_assert(N2 % 16 == 0 && N2 <= 256, "MMA N of the fused GEMM");
    static_assert(PIN % 2 == 0 || PAIR, "K planes come in pairs");
    static_assert(EPI != EPI_UP || P2 % 2 == 0, "fused GEMM K planes come in pairs");
    static_assert(EPI != EPI_FINAL || ((COUT == kC0 || COUT == kC0Max) && (!PAIRED || COUT == kC0)),
                  "final conv reads c0 channels");
    static_assert(TMEM_COLS <= 512, "TMEM columns");
    static_assert(OFF_PAR % 16 == 0 && COUT % 4 == 0 && N2 % 4 == 0, "parameters read as float4");
    static_assert(OFF_X % 16 == 0, "paired exchange in float4");
    static_assert(STAGES >= 2 && STAGES <= 6, "stages");
    static_assert(NB >= 2 && NB <= 4, "accumulator buffers");
    static_assert(!PAIRED || (!PAIR && PIN % 2 == 0 && 2 * COUT <= 256 && EPI != EPI_POOL &&
                              (EWG <= 2 || EPI == EPI_UP)),
                  "tap pairing");
    static_assert(SMEM <= 227 * 1024, "shared memory");
    static_assert(NSPLIT == 1 || ((EPI == EPI_STORE || EPI == EPI_CONVT) && !DYN && !SEQ),
                  "split layers: plain stores or the ConvT GEMM, static tiles, whole events");
    static_assert(EPI != EPI_CONVT || (COUT % (CUP ? CUP : 1) == 0 && (2 / NSPLIT) * CUP == COUT && !PAIR && CB == 0),
                  "ConvT GEMM: N = the part's r values x CUP");
    // the pool pairs lanes m, m + 1 as positions j, j + 1 of one sequence: even SEQ and LSEQ
    static_assert(!SEQ || (L == kSlices * SEQ - kPad &&
                           (EPI != EPI_POOL || (SEQ % 2 == 0 && LSEQ % 2 == 0))),
                  "per-interval geometry");
    static_assert(EPI != EPI_UP || CUP % 16 == 0, "16-column epilogue chunks");
    static_assert(EWG == 1 || (EWG == 2 && EPI != EPI_FINAL && EPI_COLS % 16 == 0) ||
                  (EWG == 4 && EPI == EPI_UP && (COUT / 2) % 16 == 0 && (N2 / 2) % 16 == 0),
                  "epilogue warpgroups");
    static_assert(EPI != EPI_UP || N2 % 16 == 0, "ConvT columns in 16-column chunks");
};

struct TcArgs {
    const unsigned char *inA, *inB;     // plane-major inputs (inB: skip half of the concat)
    unsigned char *out, *outp;          // conv or ConvT output; pooled output
    float *logits;                      // EPI_FINAL: [n_events][L] float32
    const unsigned char *w, *w2;        // packed weights (shared-memory image)
    const float *bias, *bias2;          // float32 biases
    const float *cs, *cs2;              // fp8: per-column dequantisation scales; 16-bit: null
    const float *final_w;               // EPI_FINAL: W[t][ci] then b (float32)
    float out_inv, mid_inv;             // fp8: 1 / scale of the stored output and of A2
    float *amax;                        // calibration: running max |x| per scale slot, or null
    int amax_out, amax_mid;             // slots of the stored output and of A2 (kScale*)
    int n_events;                       // events of the launch (its capacity with n_dyn)
    int32_t *status;
    int32_t *sched;                     // [2]: next tile, finished CTAs (zero between launches)
    const int32_t *n_dyn;               // nullable: device-side event count of the call
    int dyn_base;                       // index of the launch's first event in the call
    uint32_t stall_test_us;             // tests of the bounded waits only (0 otherwise): the
                                        // MMA thread first waits this long on a barrier that
                                        // nothing arrives on, then the kernel unwinds
};

// Calibration: folds max |v| of 16 values (rows with valid = false count as 0) into the
// warp maximum and lane 0 raises amax[slot] with an integer atomicMax on the float bits,
// which orders non-negative floats correctly and does not depend on arrival order.
__device__ __forceinline__ void amax_fold(float *amax, int slot, const float (&v)[16], bool valid) {
    float m = 0.0f;
#pragma unroll
    for (int j = 0; j < 16; ++j) m = fmaxf(m, fabsf(v[j]));
    if (!valid) m = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(amax + slot), __float_as_int(m));
}

// Barrier slots in shared memory (uint64 each). TFULL/TEMPTY/T2FULL follow the NB
// accumulator buffers (tile i: buffer i % NB), so none of them can complete a second
// phase before its waiters have seen the first; A2FULL/GREADY follow the two
// shared-memory buffers of the fused ConvT operand and of the final conv's exchange
// (tile i: i % 2).
constexpr int kRing = 12;    // tile-index ring: >= STAGES + NB tiles in flight
template <class C> struct Bars {
    static constexpr int W = 0, FULL = 1, EMPTY = 1 + C::STAGES, TFULL = 1 + 2 * C::STAGES,
                         TEMPTY = TFULL + C::NB, T2FULL = TEMPTY + C::NB, A2FULL = T2FULL + C::NB,
                         DRAIN = A2FULL + 2, GREADY = DRAIN + 1, XREADY = GREADY + 2,
                         TIDF = XREADY + 2, TIDE = TIDF + kRing, NEVER = TIDE + kRing, N = NEVER + 1;
    // after the barriers: TMEM address slot, abort flag, then the ring of tile indices
    static constexpr int RING_OFF = N * 8 + 16;
    static_assert(RING_OFF + 4 * kRing <= 512, "barrier area");
    static_assert(kRing >= C::STAGES + C::NB, "ring depth");
};

template <class C>
__device__ __forceinline__ void tile_pos(int t, int &e, int &p0) {
    e = t / C::TPE;
    const int k = t % C::TPE;
    p0 = C::EPI == EPI_FINAL ? k * C::STRIDE - kPad : k * C::STRIDE;
}

// Per-interval layout: position p of the event lies in sequence s at position j of it;
// j = -2 or -1 is one of the two zero rows before sequence s. Whole events: s = 0, j = p.
template <class C>
__device__ __forceinline__ void seq_pos(int p, int &s, int &j) {
    if constexpr (C::SEQ != 0) {
        s = (p + kPad) / C::SEQ;
        j = (p + kPad) % C::SEQ - kPad;
    } else {
        s = 0;
        j = p;
    }
}

// Quantises 16 values to the form's element type and stores them as 16 / PW plane rows.
template <int PREC>
__device__ __forceinline__ void put16(unsigned char *p0, size_t plane_stride, const float (&v)[16],
                                      float inv) {
    if constexpr (is16(PREC)) {
        using T = typename Elem<PREC>::T;
        *reinterpret_cast<uint4 *>(p0) = pack8<T>(v);
        *reinterpret_cast<uint4 *>(p0 + plane_stride) = pack8<T>(v + 8);
    } else {
        uint4 pk;
        pack_e4m3<16>(v, inv, reinterpret_cast<uint32_t *>(&pk));
        *reinterpret_cast<uint4 *>(p0) = pk;
    }
}

// Zeroes storage row `row` of planes [k0, k0 + nk) of event e in a tensor of `planes` planes.
__device__ __forceinline__ void zero_planes(unsigned char *base, int64_t e, int k0, int nk, int planes,
                                            int64_t rows_e, int64_t row) {
    for (int k = k0; k < k0 + nk; ++k)
        *reinterpret_cast<uint4 *>(base + planar_off(e, k, planes, rows_e, row)) = make_uint4(0, 0, 0, 0);
}

template <class C>
__device__ bool producer(const TcArgs &a, unsigned char *smem, uint64_t *bar, volatile int *ring,
                         volatile int *abort) {
    using B = Bars<C>;
    uint64_t *wbar = bar + B::W, *full = bar + B::FULL, *empty = bar + B::EMPTY, *tidf = bar + B::TIDF,
             *tide = bar + B::TIDE;
    const int ntiles = a.n_events * C::TPE;
    mbar_arrive_expect_tx(wbar, C::W_BYTES + C::W2_BYTES);
    bulk_g2s(smem + C::OFF_W, a.w + (size_t)((int)blockIdx.x % C::NSPLIT) * C::W_BYTES, C::W_BYTES, wbar);
    if (C::W2_BYTES) bulk_g2s(smem + C::OFF_W2, a.w2, C::W2_BYTES, wbar);
    int i = 0;
    bool ok = true;
    // DYN: one tile index ahead, so the atomic's latency overlaps a tile; else a stride
    int t_next = C::DYN ? atomicAdd(a.sched, 1) : (int)blockIdx.x / C::NSPLIT;
    for (;; ++i) {
        const int t = t_next < ntiles ? t_next : -1;
        if constexpr (C::DYN) {   // next tile (or -1: none left) to the MMA thread and the epilogue
            const int r = i % kRing;
            if (!mbar_wait(&tide[r], ((i / kRing) & 1) ^ 1, abort)) { ok = false; break; }
            ring[r] = t;
            mbar_arrive(&tidf[r]);
        }
        if (t < 0) break;
        t_next = C::DYN ? atomicAdd(a.sched, 1) : t + (int)gridDim.x / C::NSPLIT;
        const int s = i % C::STAGES;
        const uint32_t ph = (i / C::STAGES) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1, abort)) { ok = false; break; }
        int e, p0;
        tile_pos<C>(t, e, p0);
        // tile row r <-> storage row p0 + ROW_OFF + r; rows before the event start are not copied
        const int src0 = p0 + C::ROW_OFF > 0 ? p0 + C::ROW_OFF : 0, dst0 = src0 - p0 - C::ROW_OFF;
        const int rows = min(C::ROWS - dst0, C::ROWS_E - src0);
        unsigned char *dst = smem + C::OFF_A + s * C::A_STAGE + dst0 * 16;
        if constexpr (C::PAIR) {
            // the zero-weight 6th tap reads one row past the copied ones on an event's last
            // tile; 0 x (stale bits of a NaN) would be NaN, so that row is zeroed first
            if (dst0 + rows < C::ROWS) {
                for (int k = 0; k < C::PIN; ++k)
                    *reinterpret_cast<uint4 *>(dst + k * C::ROWS * 16 + rows * 16) = make_uint4(0, 0, 0, 0);
                fence_proxy_async_smem();
            }
        }
        mbar_arrive_expect_tx(&full[s], (uint32_t)(C::PIN * rows * 16));
        for (int k = 0; k < C::PA; ++k)
            bulk_g2s(dst + k * C::ROWS * 16, a.inA + planar_off(e, k, C::PA, C::ROWS_E, src0), rows * 16,
                     &full[s]);
        for (int k = 0; k < C::PB; ++k)
            bulk_g2s(dst + (C::PA + k) * C::ROWS * 16, a.inB + planar_off(e, k, C::PB, C::ROWS_E, src0),
                     rows * 16, &full[s]);
    }
    // copies still in flight land before the CTA can exit: wait (bounded) for the last ones
    for (int j = max(0, i - C::STAGES); j < i; ++j) {
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(&full[j % C::STAGES], (j / C::STAGES) & 1))
            if (globaltimer() - t0 > kWaitLimitNs) break;
    }
    if (!mbar_try_wait(wbar, 0)) {
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(wbar, 0)) if (globaltimer() - t0 > kWaitLimitNs) break;
    }
    return ok;
}

template <class C>
__device__ __forceinline__ void mma_t(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, bool acc) {
    if constexpr (is16(C::PREC)) mma_f16(d, ad, bd, idesc, acc);
    else mma_fp8(d, ad, bd, idesc, acc);
}

template <class C>
__device__ __forceinline__ void issue_conv(uint32_t d, uint32_t as, uint32_t w_base) {
    if constexpr (C::PAIRED) {
        // weights: group g (taps 2g, 2g + 1; g = 2: tap 4) at w_base + g * GROUP, planes of N_g rows
        constexpr uint32_t N01 = 2 * C::COUT, GROUP = C::PIN * N01 * 16;
        constexpr uint32_t ID01 = idesc_f32acc(kTileM, N01, C::FMT), ID4 = idesc_f32acc(kTileM, C::COUT, C::FMT);
#pragma unroll
        for (int kb = 0; kb < C::PIN / 2; ++kb) {
            const uint32_t a = as + 2 * kb * C::ROWS * 16;
#pragma unroll
            for (int g = 0; g < 2; ++g)
                mma_t<C>(d, smem_desc(a + 2 * g * 16, C::ROWS * 16, 128),
                         smem_desc(w_base + g * GROUP + 2 * kb * N01 * 16, N01 * 16, 128), ID01, (kb | g) != 0);
            mma_t<C>(d, smem_desc(a + 4 * 16, C::ROWS * 16, 128),
                     smem_desc(w_base + 2 * GROUP + 2 * kb * C::COUT * 16, C::COUT * 16, 128), ID4, true);
        }
    } else if constexpr (C::PAIR) {
#pragma unroll
        for (int j = 0; j < C::TAPS / 2; ++j) {
            const uint64_t ad = smem_desc(as + 2 * j * 16, 16, 128);
            const uint64_t bd = smem_desc(w_base + 2 * j * C::COUT * 16, C::COUT * 16, 128);
            mma_t<C>(d, ad, bd, C::IDESC1, j != 0);
        }
    } else {
#pragma unroll
        for (int tap = 0; tap < C::TAPS; ++tap)
#pragma unroll
            for (int kb = 0; kb < C::PIN / 2; ++kb) {
                const uint64_t ad = smem_desc(as + 2 * kb * C::ROWS * 16 + tap * 16, C::ROWS * 16, 128);
                const uint64_t bd = smem_desc(w_base + (tap * C::PIN + 2 * kb) * C::COUT * 16,
                                              C::COUT * 16, 128);
                mma_t<C>(d, ad, bd, C::IDESC1, (tap | kb) != 0);
            }
    }
}

template <class C>
__device__ __forceinline__ void issue_up(uint32_t d2, uint32_t a2, uint32_t w2_base) {
#pragma unroll
    for (int kb = 0; kb < C::P2 / 2; ++kb) {
        const uint64_t ad = smem_desc(a2 + 2 * kb * kTileM * 16, kTileM * 16, 128);
        const uint64_t bd = smem_desc(w2_base + 2 * kb * C::N2 * 16, C::N2 * 16, 128);
        mma_t<C>(d2, ad, bd, C::IDESC2, kb != 0);
    }
}

// The fused ConvT with its A operand in tensor memory (A2T): the K step kb reads the 8
// columns holding channels [16 kb, 16 kb + 16) (16-bit; 32 e4m3 channels per step).
template <class C>
__device__ __forceinline__ void issue_up_ts(uint32_t d2, uint32_t a2_tmem, uint32_t w2_base) {
#pragma unroll
    for (int kb = 0; kb < C::P2 / 2; ++kb) {
        const uint64_t bd = smem_desc(w2_base + 2 * kb * C::N2 * 16, C::N2 * 16, 128);
        if constexpr (is16(C::PREC)) mma_f16_ts(d2, a2_tmem + 8 * kb, bd, C::IDESC2, kb != 0);
        else mma_fp8_ts(d2, a2_tmem + 8 * kb, bd, C::IDESC2, kb != 0);
    }
}

template <class C>
__device__ __forceinline__ void issue_up_any(uint32_t tmem, int bp, int ap, uint32_t a2_base, uint32_t w2_base) {
    if constexpr (C::A2T)
        issue_up_ts<C>(tmem + bp * C::COLS_BUF + C::UP_OFF, tmem + C::A2_COL0 + ap * C::A2_COLS, w2_base);
    else
        issue_up<C>(tmem + bp * C::COLS_BUF + C::UP_OFF, a2_base + ap * C::A2_BYTES, w2_base);
}

// One thread issues all MMAs. With a fused ConvT, the conv of tile i is issued before the
// ConvT of tile i - 1, so the tensor core works while the epilogue turns tile i - 1's
// conv accumulator into the shared-memory operand of its ConvT.
template <class C>
__device__ bool mma_issuer(const TcArgs &a, unsigned char *smem, uint64_t *bar, uint32_t tmem,
                           volatile int *ring, volatile int *abort) {
    using B = Bars<C>;
    uint64_t *wbar = bar + B::W, *full = bar + B::FULL, *empty = bar + B::EMPTY,
             *tfull = bar + B::TFULL, *tempty = bar + B::TEMPTY, *a2full = bar + B::A2FULL,
             *t2full = bar + B::T2FULL, *drain = bar + B::DRAIN, *tidf = bar + B::TIDF, *tide = bar + B::TIDE;
    bool ok = mbar_wait(wbar, 0, abort);
    tc_fence_after();
    const uint32_t a_base = smem_u32(smem + C::OFF_A);
    const uint32_t w_base = smem_u32(smem + C::OFF_W);
    const uint32_t w2_base = smem_u32(smem + C::OFF_W2);
    const uint32_t a2_base = smem_u32(smem + C::OFF_A2);
    const int ntiles = a.n_events * C::TPE;
    int i = 0;
    for (; ok; ++i) {
        if constexpr (C::DYN) {
            const int r = i % kRing;
            if (!mbar_wait(&tidf[r], (i / kRing) & 1, abort)) { ok = false; break; }
            const int t = ring[r];
            mbar_arrive(&tide[r]);
            if (t < 0) break;
        } else if ((int)blockIdx.x / C::NSPLIT + i * ((int)gridDim.x / C::NSPLIT) >= ntiles) {
            break;
        }
        const int s = i % C::STAGES, b = i % C::NB;
        const uint32_t ph_s = (i / C::STAGES) & 1, ph_b = (i / C::NB) & 1;
        if (!mbar_wait(&tempty[b], ph_b ^ 1, abort) || !mbar_wait(&full[s], ph_s, abort)) { ok = false; break; }
        tc_fence_after();
        issue_conv<C>(tmem + b * C::COLS_BUF, a_base + s * C::A_STAGE, w_base);
        mma_commit(&empty[s]);
        mma_commit(&tfull[b]);
        if constexpr (C::EPI == EPI_UP) {
            if (i > 0) {
                const int bp = (i - 1) % C::NB, ap = (i - 1) & 1;
                if (!mbar_wait(&a2full[ap], ((i - 1) >> 1) & 1, abort)) { ok = false; break; }
                tc_fence_after();
                issue_up_any<C>(tmem, bp, ap, a2_base, w2_base);
                mma_commit(&t2full[bp]);
            }
        }
    }
    if constexpr (C::EPI == EPI_UP) {
        if (ok && i > 0) {
            const int bp = (i - 1) % C::NB, ap = (i - 1) & 1;
            if (mbar_wait(&a2full[ap], ((i - 1) >> 1) & 1, abort)) {
                tc_fence_after();
                issue_up_any<C>(tmem, bp, ap, a2_base, w2_base);
                mma_commit(&t2full[bp]);
            } else {
                ok = false;
            }
        }
    }
    // every MMA issued above completes before TMEM is released
    mma_commit(drain);
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(drain, 0)) if (globaltimer() - t0 > kWaitLimitNs) break;
    return ok;
}

// 16 consecutive parameters from shared memory in four 16-byte loads (p 16-byte aligned):
// the epilogues read their biases, scales and final-conv weights per tile, and scalar
// broadcast loads made the shared-memory pipe the bottleneck of the final conv.
__device__ __forceinline__ void lds16(const float *p, float (&v)[16]) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 x = q[i];
        v[4 * i] = x.x; v[4 * i + 1] = x.y; v[4 * i + 2] = x.z; v[4 * i + 3] = x.w;
    }
}

// Paired taps: conv columns [c0, c0 + W) of row m = E[m] + O[m + 1]. The O columns are
// loaded first: lane 0 of each quarter publishes its O row into sx and arrives on xready
// (`use`: how many times this barrier completed before, for its parity); O[m + 1] then
// comes from the next lane, or for lane 31 from the next quarter's published row. With
// several column chunks per tile (MANY) the E columns load while the conv epilogue's
// threads meet; with one, E and O load together after the meeting (each measured the
// faster of the two orders: dec3_up2 96.1 -> 92.5 us, dec2_up1 74.8 vs 76.4 us).
// Returns false on a timed-out wait.
template <class C, int W, bool MANY>
__device__ __forceinline__ bool paired_cols(uint32_t dcol, int c0, float *sx, int q, int lane,
                                            uint64_t *xready, uint32_t use, volatile int *abort,
                                            float (&v)[W]) {
    float o[W];
    if constexpr (W == 32) tmem_ld32(dcol + C::COUT + c0, o);
    else tmem_ld16(dcol + C::COUT + c0, o);
    if (lane == 0) {
        float4 *d4 = reinterpret_cast<float4 *>(sx + q * C::COUT + c0);
#pragma unroll
        for (int j4 = 0; j4 < W / 4; ++j4)
            d4[j4] = make_float4(o[4 * j4], o[4 * j4 + 1], o[4 * j4 + 2], o[4 * j4 + 3]);
    }
    mbar_arrive(xready);
    if constexpr (MANY) {
        if constexpr (W == 32) tmem_ld32(dcol + c0, v);
        else tmem_ld16(dcol + c0, v);
        if (!mbar_wait(xready, use & 1u, abort)) return false;
    } else {
        if (!mbar_wait(xready, use & 1u, abort)) return false;
        if constexpr (W == 32) tmem_ld32x2(dcol + c0, dcol + C::COUT + c0, v, o);
        else tmem_ld16x2(dcol + c0, dcol + C::COUT + c0, v, o);
    }
#pragma unroll
    for (int j = 0; j < W; ++j) o[j] = __shfl_down_sync(0xffffffffu, o[j], 1);
    if (lane == 31) {     // row 32 q + 31: its O[m + 1] is the next quarter's first row
        const float4 *n4 = reinterpret_cast<const float4 *>(sx + (q + 1) * C::COUT + c0);
#pragma unroll
        for (int j4 = 0; j4 < W / 4; ++j4) {
            const float4 x = q < 3 ? n4[j4] : make_float4(0.f, 0.f, 0.f, 0.f);
            o[4 * j4] = x.x; o[4 * j4 + 1] = x.y; o[4 * j4 + 2] = x.z; o[4 * j4 + 3] = x.w;
        }
    }
#pragma unroll
    for (int j = 0; j < W; ++j) v[j] += o[j];
    return true;
}

// Epilogue pieces, one TMEM lane (tile row m, position p) per thread.
// Conv columns [c_beg, c_beg + NC) of accumulator dcol: bias, LeakyReLU, then either the
// fused ConvT's shared-memory operand (A2) or the stored output (+ the 2:1 max-pool).
// inseq: the row is a position of a sequence (false: a zero row between sequences of the
// per-interval layout, stored as zeros). Paired taps: the exchange of each column chunk
// meets on xready, which completed xuse0 times before this tile (returns false on a
// timed-out wait).
template <class C, int NC>
__device__ __forceinline__ bool epi_conv(const TcArgs &a, unsigned char *smem, const float *sbias,
                                         const float *scs, uint32_t dcol, int c_beg, int ab, int e,
                                         int p, int m, bool valid, float *sx = nullptr,
                                         uint32_t a2t = 0, bool inseq = true, uint64_t *xready = nullptr,
                                         uint32_t xuse0 = 0, volatile int *abort = nullptr) {
    constexpr int64_t ROWS_P = C::ROWS_P;
    int sq, jq;
    seq_pos<C>(p, sq, jq);
    // pooled row: position j / 2 of sequence s (whole events: p / 2)
    const int64_t prow = C::SEQ ? (int64_t)sq * C::SEQP + jq / 2 + kPad : p / 2 + kPad;
    constexpr int LDW = C::ldw(NC);
#pragma unroll 1
    for (int cc = 0; cc < NC; cc += LDW) {
        float vv[LDW];
        if constexpr (C::PAIRED) {
            if (!paired_cols<C, LDW, (NC > LDW)>(dcol, c_beg + cc, sx, m >> 5, m & 31, xready, xuse0 + cc / LDW,
                                                 abort, vv))
                return false;
        } else if constexpr (LDW == 32) {
            tmem_ld32(dcol + c_beg + cc, vv);
        } else {
            tmem_ld16(dcol + c_beg + cc, vv);
        }
#pragma unroll
        for (int h = 0; h < LDW / 16; ++h) {
            const int c0 = c_beg + cc + 16 * h;
            float v[16], bj[16];
            lds16(sbias + c0, bj);
            if constexpr (is16(C::PREC)) {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = leaky(vv[16 * h + j] + bj[j]);
            } else {
                float sc[16];
                lds16(scs + c0, sc);
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = leaky(fmaf(vv[16 * h + j], sc[j], bj[j]));
            }
            if constexpr (C::SEQ != 0) {
                if (!inseq) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = 0.0f;
                }
            }
            if constexpr (C::EPI == EPI_UP && C::A2T) {
                // this row's 16 channels into its TMEM lane: 16-bit pairs (8 columns) or
                // e4m3 quads (4 columns), the K order the MMA reads
                if (a.amax) amax_fold(a.amax, a.amax_mid, v, valid);
                if constexpr (is16(C::PREC)) {
                    using T = typename Elem<C::PREC>::T;
                    uint32_t r[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) r[j] = pack2<T>(v[2 * j], v[2 * j + 1]);
                    tmem_st<8>(a2t + c0 / 2, r);
                } else {
                    uint32_t r[4];
                    pack_e4m3<16>(v, a.mid_inv, r);
                    tmem_st<4>(a2t + c0 / 4, r);
                }
            } else if constexpr (C::EPI == EPI_UP) {
                if (a.amax) amax_fold(a.amax, a.amax_mid, v, valid);
                unsigned char *a2 = smem + C::OFF_A2 + ab * C::A2_BYTES;
                put16<C::PREC>(a2 + ((c0 / C::PW) * kTileM + m) * 16, (size_t)kTileM * 16, v, a.mid_inv);
            } else {
                if (a.amax) amax_fold(a.amax, a.amax_out, v, valid);
                if (valid)   // a split layer's part writes its own planes of the output
                    put16<C::PREC>(a.out + planar_off(e, ((int)blockIdx.x % C::NSPLIT) * C::POUT + c0 / C::PW,
                                                      C::POUT_TOT, C::ROWS_E, p + kPad),
                              (size_t)C::ROWS_E * 16, v, a.out_inv);
                if constexpr (C::EPI == EPI_POOL) {
                    float w[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) w[j] = fmaxf(v[j], __shfl_xor_sync(0xffffffffu, v[j], 1));
                    if (valid && inseq && (m & 1) == 0)
                        put16<C::PREC>(a.outp + planar_off(e, c0 / C::PW, C::POUT, ROWS_P, prow),
                                  (size_t)ROWS_P * 16, w, a.out_inv);
                }
            }
        }
    }
    return true;
}

// Fused ConvT columns [n_beg, n_beg + NC) (n = r * CUP + co: output row 2p + r, channel
// co): bias, LeakyReLU, store; the thread of p = 0 / L - 1 (with pads) zeroes the pads.
// r0: the first output-row parity of these columns (the ConvT GEMM split by r: its part).
template <class C, int NC>
__device__ __forceinline__ void epi_up(const TcArgs &a, const float *sbias2, const float *scs2,
                                       uint32_t dcol, int n_beg, int e, int p, bool valid, bool pads,
                                       int r0 = 0) {
    constexpr int LO = 2 * C::L;
    constexpr int64_t ROWS_O = C::ROWS_O;
    int sq, jq;
    seq_pos<C>(p, sq, jq);
    const bool inseq = !C::SEQ || (jq >= 0 && jq < C::LSEQ);
    // output rows 2 j + r of sequence s (whole events: 2 p + r)
    const int64_t orow0 = C::SEQ ? (int64_t)sq * C::SEQU + 2 * jq + kPad : 2 * p + kPad;
    constexpr int PUP = C::CUP / C::PW;
    constexpr int LDW = NC % 32 == 0 ? 32 : 16;
#pragma unroll 1
    for (int cc = 0; cc < NC; cc += LDW) {
        float vv[LDW];
        if constexpr (LDW == 32) {
            tmem_ld32(dcol + C::UP_OFF + n_beg + cc, vv);
        } else {
            tmem_ld16(dcol + C::UP_OFF + n_beg + cc, vv);
        }
#pragma unroll
        for (int h = 0; h < LDW / 16; ++h) {
            const int c0 = n_beg + cc + 16 * h;
            const int r = r0 + c0 / C::CUP, co0 = c0 % C::CUP;
            float v[16], bj[16];
            lds16(sbias2 + co0, bj);
            if constexpr (is16(C::PREC)) {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = leaky(vv[16 * h + j] + bj[j]);
            } else {
                float sc[16];
                lds16(scs2 + c0, sc);
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = leaky(fmaf(vv[16 * h + j], sc[j], bj[j]));
            }
            if (a.amax) amax_fold(a.amax, a.amax_out, v, valid && inseq);
            if (valid && inseq)
                put16<C::PREC>(a.out + planar_off(e, co0 / C::PW, PUP, ROWS_O, orow0 + r),
                          (size_t)ROWS_O * 16, v, a.out_inv);
        }
    }
    if constexpr (C::SEQ != 0) {     // each output sequence's zero rows
        if (pads && valid && jq == 0) {
            zero_planes(a.out, e, 0, PUP, PUP, ROWS_O, (int64_t)sq * C::SEQU);
            zero_planes(a.out, e, 0, PUP, PUP, ROWS_O, (int64_t)sq * C::SEQU + 1);
        }
        if (pads && valid && jq == C::LSEQ - 1 && sq == kSlices - 1) {   // the event's last two rows
            zero_planes(a.out, e, 0, PUP, PUP, ROWS_O, (int64_t)kSlices * C::SEQU);
            zero_planes(a.out, e, 0, PUP, PUP, ROWS_O, (int64_t)kSlices * C::SEQU + 1);
        }
    } else {
        if (pads && p == 0) {
            zero_planes(a.out, e, 0, PUP, PUP, ROWS_O, 0);
            zero_planes(a.out, e, 0, PUP, PUP, ROWS_O, 1);
        }
        if (pads && p == C::L - 1) {
            zero_planes(a.out, e, 0, PUP, PUP, ROWS_O, LO + kPad);
            zero_planes(a.out, e, 0, PUP, PUP, ROWS_O, LO + kPad + 1);
        }
    }
}

template <class C>
__device__ bool epilogue(const TcArgs &a, unsigned char *smem, uint64_t *bar, uint32_t tmem,
                         volatile int *ring, volatile int *abort, int warp, int lane) {
    using B = Bars<C>;
    uint64_t *tfull = bar + B::TFULL, *tempty = bar + B::TEMPTY, *a2full = bar + B::A2FULL,
             *t2full = bar + B::T2FULL, *gready = bar + B::GREADY, *xready = bar + B::XREADY,
             *tidf = bar + B::TIDF, *tide = bar + B::TIDE;
    const float *par = reinterpret_cast<const float *>(smem + C::OFF_PAR);
    const float *sbias = par, *sbias2 = par + C::COUT, *scs = par + C::COUT + C::N2,
                *scs2 = scs + C::COUT, *sfin = par + 2 * (C::COUT + C::N2);
    const int q = warp & 3;                         // TMEM lane quarter of this warp
    const int m = q * 32 + lane;                    // tile row
    const int wg = (warp - 2) >> 2;                 // epilogue warpgroup
    const uint32_t lane_field = (uint32_t)(q * 32) << 16;
    const uint32_t a2_lane = tmem + lane_field + C::A2_COL0;    // A2T: this warp's lanes of the A2 buffers
    constexpr int64_t ROWS_P = C::ROWS_P;           // pooled tensor
    constexpr bool ROLES = C::EPI == EPI_UP && C::EWG >= 2;
    const int ntiles = a.n_events * C::TPE;
    const int part = (int)blockIdx.x % C::NSPLIT;   // this CTA's part of a split layer
    for (int i = 0;; ++i) {
        int t = (int)blockIdx.x / C::NSPLIT + i * ((int)gridDim.x / C::NSPLIT);
        if constexpr (C::DYN) {
            const int r = i % kRing;
            if (!mbar_wait(&tidf[r], (i / kRing) & 1, abort)) return false;
            t = ring[r];
            __syncwarp();
            if (lane == 0) mbar_arrive(&tide[r]);
            if (t < 0) break;
        } else if (t >= ntiles) {
            break;
        }
        const int b = i % C::NB, ab = i & 1;
        const uint32_t ph_b = (i / C::NB) & 1, ph_a = (i >> 1) & 1;
        int e, p0;
        tile_pos<C>(t, e, p0);
        const int p = p0 + m;
        // rows past the stride belong to the next tile (and row 127 of a paired tile is incomplete)
        const bool valid = p >= 0 && p < C::L && m < C::ROWS_OK;
        int sq, jq;                                 // per-interval layout: sequence, position
        seq_pos<C>(p, sq, jq);
        const bool inseq = !C::SEQ || (jq >= 0 && jq < C::LSEQ);
        const uint32_t dcol = tmem + lane_field + b * C::COLS_BUF;
        float *sx = reinterpret_cast<float *>(smem + C::OFF_X) + ab * 4 * C::COUT;
        if constexpr (ROLES) {
            constexpr int PER = C::EWG / 2;                 // warpgroups per role
            const int part = wg % PER;
            if (wg < PER) {     // conv accumulator -> ConvT operand
                if (!mbar_wait(&tfull[b], ph_b, abort)) return false;
                tc_fence_after();
                if (!epi_conv<C, C::COUT / PER>(a, smem, sbias, scs, dcol, part * (C::COUT / PER), ab, e, p, m,
                                                valid, sx, a2_lane + ab * C::A2_COLS, inseq, &xready[ab],
                                                (uint32_t)(i >> 1) * C::xchunks(C::COUT / PER), abort))
                    return false;
                if constexpr (C::A2T) tmem_st_wait();   // A2 in TMEM complete before the MMA reads it
                else fence_proxy_async_smem();          // A2 writes -> visible to the tensor core
                tc_fence_before();
                mbar_arrive(&a2full[ab]);
            } else {            // ConvT accumulator -> output; frees the buffer
                if (!mbar_wait(&t2full[b], ph_b, abort)) return false;
                tc_fence_after();
                epi_up<C, C::N2 / PER>(a, sbias2, scs2, dcol, part * (C::N2 / PER), e, p, valid, part == 0);
                tc_fence_before();
                mbar_arrive(&tempty[b]);
            }
            continue;
        }
        if (!mbar_wait(&tfull[b], ph_b, abort)) return false;
        tc_fence_after();
        if constexpr (C::EPI == EPI_CONVT) {   // the ConvT GEMM: this warpgroup's columns
            epi_up<C, C::EPI_COLS>(a, sbias, scs, dcol, wg * C::EPI_COLS, e, p, valid, wg == 0 && part == 0,
                                   part * (C::COUT / C::CUP));
            tc_fence_before();
            mbar_arrive(&tempty[b]);
            continue;
        }
        if constexpr (C::EPI == EPI_FINAL) {
            constexpr int NCH = C::COUT / 16;       // 16-channel chunks of d1
            float v[NCH][16];
            if constexpr (C::PAIRED) {
                if (!paired_cols<C, 16, false>(dcol, 0, sx, q, lane, &xready[ab], (uint32_t)(i >> 1), abort, v[0]))
                    return false;
            } else {
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) tmem_ld16(dcol + 16 * ch, v[ch]);
            }
            tc_fence_before();
            mbar_arrive(&tempty[b]);
            float g[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) {
                float bj[16], sc[16];
                lds16(sbias + 16 * ch, bj);
                if constexpr (is16(C::PREC)) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) sc[j] = 1.0f;
                } else {
                    lds16(scs + 16 * ch, sc);
                }
#pragma unroll
                for (int j = 0; j < 16; ++j)   // zero padding outside the event or its sequence
                    v[ch][j] = valid && inseq ? leaky(fmaf(v[ch][j], sc[j], bj[j])) : 0.0f;
                if (a.amax) amax_fold(a.amax, a.amax_out, v[ch], valid && inseq);
                // the final conv's partial sums over this chunk's channels, in channel order:
                // taps (0, 1) and (2, 3) as packed two-lane FMAs (each lane an fmaf), from
                // weights stored per channel as (w0, w1, w2, w3), then tap 4
                float2 g01 = make_float2(g[0], g[1]), g23 = make_float2(g[2], g[3]);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float4 w4 = reinterpret_cast<const float4 *>(sfin)[16 * ch + j];
                    const float2 vv = make_float2(v[ch][j], v[ch][j]);
                    g01 = __ffma2_rn(make_float2(w4.x, w4.y), vv, g01);
                    g23 = __ffma2_rn(make_float2(w4.z, w4.w), vv, g23);
                }
                g[0] = g01.x; g[1] = g01.y; g[2] = g23.x; g[3] = g23.y;
                {
                    float wf[16];
                    lds16(sfin + 4 * C::COUT + 16 * ch, wf);
                    float acc = g[4];
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc = fmaf(wf[j], v[ch][j], acc);
                    g[4] = acc;
                }
            }
            float *sg = reinterpret_cast<float *>(smem + C::OFF_G) + ab * 5 * kTileM;
#pragma unroll
            for (int tp = 0; tp < 5; ++tp) sg[tp * kTileM + m] = g[tp];
            // neighbours' partial sums: a bounded mbarrier among the 128 epilogue threads
            mbar_arrive(&gready[ab]);
            if (!mbar_wait(&gready[ab], ph_a, abort)) return false;
            // per-interval layout: the logits of an interval's bins are its sequence's
            // central positions [kIvPad, kIvPad + kSliceBins)
            const bool out = !C::SEQ || (jq >= kIvPad && jq < kIvPad + kSliceBins);
            if (m >= kPad && m < kPad + C::STRIDE && valid && out) {
                // f(p) = b + sum_t g_t(p + t - 2), in tap order
                float f = sfin[5 * C::COUT];
#pragma unroll
                for (int tp = 0; tp < 5; ++tp) f += sg[tp * kTileM + m + tp - 2];
                if constexpr (C::SEQ != 0) a.logits[(size_t)e * kBins + sq * kSliceBins + jq - kIvPad] = f;
                else a.logits[(size_t)e * C::L + p] = f;
            }
            continue;
        }
        if constexpr (C::EPI == EPI_UP) {   // one warpgroup: conv, then the ConvT
            if (!epi_conv<C, C::COUT>(a, smem, sbias, scs, dcol, 0, ab, e, p, m, valid, sx,
                                      a2_lane + ab * C::A2_COLS, inseq, &xready[ab],
                                      (uint32_t)(i >> 1) * C::xchunks(C::COUT), abort))
                return false;
            if constexpr (C::A2T) tmem_st_wait();
            else fence_proxy_async_smem();
            tc_fence_before();
            mbar_arrive(&a2full[ab]);
            if (!mbar_wait(&t2full[b], ph_b, abort)) return false;
            tc_fence_after();
            epi_up<C, C::N2>(a, sbias2, scs2, dcol, 0, e, p, valid, true);
        } else {                            // this warpgroup's conv columns
            static_assert(!C::PAIRED || C::EPI == EPI_STORE, "paired stores");
            // paired taps (the wide network's split dec3): E[m] + O[m + 1]
            if (!epi_conv<C, C::EPI_COLS>(a, smem, sbias, scs, dcol, wg * C::EPI_COLS, ab, e, p, m, valid, sx, 0,
                                          inseq, &xready[ab], (uint32_t)(i >> 1) * C::xchunks(C::EPI_COLS), abort))
                return false;
            if (wg == 0 && (p == 0 || p == C::L - 1)) {
                const int r0 = p == 0 ? 0 : C::L + kPad;
                zero_planes(a.out, e, part * C::POUT, C::POUT, C::POUT_TOT, C::ROWS_E, r0);
                zero_planes(a.out, e, part * C::POUT, C::POUT, C::POUT_TOT, C::ROWS_E, r0 + 1);
                if constexpr (C::EPI == EPI_POOL && C::SEQ == 0) {
                    const int rp = p == 0 ? 0 : C::L / 2 + kPad;
                    zero_planes(a.outp, e, 0, C::POUT, C::POUT, ROWS_P, rp);
                    zero_planes(a.outp, e, 0, C::POUT, C::POUT, ROWS_P, rp + 1);
                }
            }
            if constexpr (C::EPI == EPI_POOL && C::SEQ != 0) {   // each pooled sequence's zero rows
                // (the two before it; after the last sequence also the event's last two)
                if (wg == 0 && valid && (jq == 0 || (jq == C::LSEQ - 2 && sq == kSlices - 1))) {
                    const int64_t rp = jq == 0 ? (int64_t)sq * C::SEQP : (int64_t)kSlices * C::SEQP;
                    zero_planes(a.outp, e, 0, C::POUT, C::POUT, ROWS_P, rp);
                    zero_planes(a.outp, e, 0, C::POUT, C::POUT, ROWS_P, rp + 1);
                }
            }
        }
        tc_fence_before();
        mbar_arrive(&tempty[b]);
    }
    return true;
}

template <class C>
__global__ void __launch_bounds__(C::THREADS) __maxnreg__(C::MAXREG) k_conv_tc(TcArgs a) {
    using B = Bars<C>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + B::N);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *ring = reinterpret_cast<volatile int *>(reinterpret_cast<unsigned char *>(bar) + B::RING_OFF);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // biases, column scales and the final conv in shared memory
    float *par = reinterpret_cast<float *>(smem + C::OFF_PAR);
    const int part = (int)blockIdx.x % C::NSPLIT;   // this CTA's part of a split layer
    for (int k = threadIdx.x; k < C::NPAR; k += C::THREADS) {
        float v;
        if (k < C::COUT) v = C::EPI == EPI_CONVT ? a.bias[k % C::CUP] : a.bias[part * C::COUT + k];
        else if (k < C::COUT + C::N2) v = a.bias2[(k - C::COUT) % (C::CUP > 0 ? C::CUP : 1)];
        else if (k < 2 * C::COUT + C::N2) v = a.cs ? a.cs[part * C::COUT + k - C::COUT - C::N2] : 1.0f;
        else if (k < 2 * (C::COUT + C::N2)) v = a.cs2 ? a.cs2[k - 2 * C::COUT - C::N2] : 1.0f;
        else {   // the final conv: (w0, w1, w2, w3) per channel, then w4 per channel, then b
            const int f = k - 2 * (C::COUT + C::N2);
            v = f < 4 * C::COUT ? a.final_w[(f & 3) * C::COUT + (f >> 2)] : a.final_w[f];
        }
        par[k] = v;
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[B::W], 1);
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&bar[B::FULL + s], 1);
            mbar_init(&bar[B::EMPTY + s], 1);
        }
        for (int b = 0; b < C::NB; ++b) {
            mbar_init(&bar[B::TFULL + b], 1);
            mbar_init(&bar[B::TEMPTY + b], C::EPI == EPI_UP ? 128 * ((C::EWG + 1) / 2) : 128 * C::EWG);
            mbar_init(&bar[B::T2FULL + b], 1);
        }
        for (int b = 0; b < 2; ++b) mbar_init(&bar[B::A2FULL + b], 128 * ((C::EWG + 1) / 2));
        mbar_init(&bar[B::DRAIN], 1);
        mbar_init(&bar[B::GREADY], 128);
        mbar_init(&bar[B::GREADY + 1], 128);
        mbar_init(&bar[B::XREADY], 128 * ((C::EWG + 1) / 2));     // the conv epilogue's warpgroups
        mbar_init(&bar[B::XREADY + 1], 128 * ((C::EWG + 1) / 2));
        for (int r = 0; r < kRing; ++r) {
            mbar_init(&bar[B::TIDF + r], 1);                // the producer
            mbar_init(&bar[B::TIDE + r], 1 + 4 * C::EWG);   // the MMA thread and each epilogue warp
        }
        mbar_init(&bar[B::NEVER], 1);                       // bounded-wait tests: nobody arrives
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // the prologue above only touched weights and parameters; the activations are the
    // previous kernel's output
    grid_dep_wait();
    grid_dep_launch();
    // with a device-side count, the events of this launch are known from here on
    TcArgs r = a;
    r.n_events = launch_events(a.n_dyn, a.dyn_base, a.n_events);

    bool ok = true;
    if (warp == 0) {
        if (lane == 0) ok = producer<C>(r, smem, bar, ring, abort);
    } else if (warp == 1) {
        // a test of the bounded waits: the wait gives up after stall_test_us, before any MMA
        if (lane == 0 && a.stall_test_us)
            ok = mbar_wait(&bar[B::NEVER], 0, abort, 1000ull * a.stall_test_us);
        if (lane == 0 && ok) ok = mma_issuer<C>(r, smem, bar, tmem, ring, abort);
    } else {
        ok = epilogue<C>(r, smem, bar, tmem, ring, abort, warp, lane);
    }
    if (!ok) {
        *abort = 1;
        raise_status(a.status, PVF_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, C::TMEM_COLS);
    if (C::DYN && threadIdx.x == 0) {   // the last CTA to finish resets the counter for the next launch
        __threadfence();
        if (atomicAdd(a.sched + 1, 1) == (int)gridDim.x - 1) {
            atomicExch(a.sched, 0);
            atomicExch(a.sched + 1, 0);
        }
    }
}

// cap: the launch schedule's CTAs per SM (0 = as many as fit)
template <class C>
cudaError_t launch_conv(const TcArgs &a, cudaStream_t s, const ProfHook *prof, const char *name, int cap) {
    if (a.n_events <= 0) return cudaSuccess;
    // shared memory request padded so that the CTAs resident on one SM never ask for more
    // than the 512 TMEM columns: tcgen05.alloc would otherwise wait for a neighbour
    constexpr int kMaxByTmem = 512 / C::TMEM_COLS;
    constexpr int kSmemPerSm = 228 * 1024;
    int smem = C::SMEM;
    const int by_tmem_smem = kSmemPerSm / kMaxByTmem - 1024;
    if (smem < by_tmem_smem) smem = by_tmem_smem;
    if (smem > 227 * 1024) smem = 227 * 1024;
    int sms = 0;
    cudaFuncAttributes fa;
    cudaError_t err = current_device_sms(&sms);
    if (err == cudaSuccess) err = prepare_kernel((const void *)k_conv_tc<C>, (size_t)smem, &fa);
    if (err != cudaSuccess) return err;
    // resident CTAs per SM: registers (each of the 4 sub-partitions holds 16K, allocated
    // per warp in units of 256), shared memory (+1 KB reserved per CTA), threads, TMEM
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = 4 * (16384 / warp_regs) / (C::THREADS / 32);
    const int by_smem = kSmemPerSm / (smem + 1024);
    const int by_threads = 2048 / C::THREADS;
    int per_sm = by_regs < by_smem ? by_regs : by_smem;
    if (by_threads < per_sm) per_sm = by_threads;
    if (kMaxByTmem < per_sm) per_sm = kMaxByTmem;
    if (cap > 0 && cap < per_sm) per_sm = cap;
    if (per_sm < 1) per_sm = 1;
    const int ntiles = a.n_events * C::TPE;
    int grid = sms * per_sm;
    if (grid > ntiles * C::NSPLIT) grid = ntiles * C::NSPLIT;
    grid = grid / C::NSPLIT * C::NSPLIT;             // every part gets the same CTAs
    if (grid < C::NSPLIT) grid = C::NSPLIT;
    ProfScope ps(prof, name, s);
    return launch_pdl(k_conv_tc<C>, dim3(grid), dim3(C::THREADS), (size_t)smem, s, a);
}

// ---------------------------------------------------------------- weight packing (host)

// Conv layers (0..5: enc2, enc3, enc4, dec3, dec2, dec1) whose taps are stacked in pairs
// along N: where it measured faster, the 16-bit dec3 (44 -> 28 MMAs per tile) and dec2. The
// FP8 form already halves the MMAs (K = 32) and measured slower paired; dec1 is bound by
// its epilogue.
constexpr bool conv_paired(int li, int prec) { return (li == 3 || li == 4) && is16(prec); }

template <int PREC> struct Net {
    using Enc2 = Cfg<PREC, 16, 0, 32, 2000, EPI_POOL, 0, 4, 1, 56, 2, false, true>;    // 6 CTAs per SM
    using Enc3 = Cfg<PREC, 32, 0, 64, 1000, EPI_POOL, 0, 4, 1, 80, 2, false, true>;    // 4
    // the fused-ConvT kernels keep the ConvT operand in TMEM (three accumulator buffers
    // leave room for its two buffers): 59 -> 55, 99 -> 96 and 77 -> 75 us (16-bit forms)
    using Enc4Up3 = Cfg<PREC, 64, 0, 128, 500, EPI_UP, 64, is16(PREC) ? 2 : 4,
                        is16(PREC) ? 2 : 4, 96, 3, false, false, true>;              // 1
    using Dec3Up2 = Cfg<PREC, 64, 64, 64, 1000, EPI_UP, 32, 3, 2, 128, 3, conv_paired(3, PREC), false,
                        true>;                                                         // 1 CTA/SM
    using Dec2Up1 = Cfg<PREC, 32, 32, 32, 2000, EPI_UP, 16, 3, 2, 128, 3, conv_paired(4, PREC), false,
                        true>;                                                         // 2
    using Dec1Final = Cfg<PREC, 16, 16, 16, 4000, EPI_FINAL, 0, 3, 1, 64, 4, conv_paired(5, PREC)>; // 5
};

// The per-interval layout (§3's batch of 40 intervals, each its own sequence of kIvLen =
// 104 positions): the same kernels over each event's 40 sequences laid end to end, with
// levels of 104, 52, 26 and 13 positions per sequence (108, 56, 30 and 17 storage rows).
template <int PREC> struct NetIv {
    static constexpr int S0 = kIvLen + kPad, S1 = kIvLen / 2 + kPad, S2 = kIvLen / 4 + kPad,
                         S3 = kIvLen / 8 + kPad;
    static constexpr int L0 = kSlices * S0 - kPad, L1 = kSlices * S1 - kPad, L2 = kSlices * S2 - kPad,
                         L3 = kSlices * S3 - kPad;
    using Enc2 = Cfg<PREC, 16, 0, 32, L1, EPI_POOL, 0, 4, 1, 56, 2, false, true, false, S1>;
    using Enc3 = Cfg<PREC, 32, 0, 64, L2, EPI_POOL, 0, 4, 1, 80, 2, false, true, false, S2>;
    using Enc4Up3 = Cfg<PREC, 64, 0, 128, L3, EPI_UP, 64, is16(PREC) ? 2 : 4, is16(PREC) ? 2 : 4, 96, 3, false,
                        false, true, S3>;
    using Dec3Up2 = Cfg<PREC, 64, 64, 64, L2, EPI_UP, 32, 3, 2, 128, 3, conv_paired(3, PREC), false, true, S2>;
    using Dec2Up1 = Cfg<PREC, 32, 32, 32, L1, EPI_UP, 16, 3, 2, 128, 3, conv_paired(4, PREC), false, true, S1>;
    using Dec1Final = Cfg<PREC, 16, 16, 16, L0, EPI_FINAL, 0, 3, 1, 64, 4, conv_paired(5, PREC), false, false,
                          S0>;
};

// The wide network (base width 32: 32/64/128/256 channels, §5's channel-count axis). The
// enc4 (128 -> 256) and dec3 (256 -> 128) weight images (320 KB in 16 bits) exceed a CTA's
// shared memory, so their output channels are split over CTA groups (parts of 64 or 32
// channels in 16 bits, 128 or 64 in e4m3), they store e4 and d3, and their ConvTs run as
// GEMM kernels of their own (up3 split by output-row parity r). dec2 + up1 has the shapes of
// the narrow network's dec3 + up2.
template <int PREC> struct Net32 {
    static constexpr int SP = is16(PREC) ? 4 : 2;            // parts of enc4 and dec3
    using Enc2 = Cfg<PREC, 32, 0, 64, 2000, EPI_POOL, 0, 4, 1, 80, 2, false, true>;
    using Enc3 = Cfg<PREC, 64, 0, 128, 1000, EPI_POOL, 0, 3, 2, 128, 2, false, true>;
    using Enc4 = Cfg<PREC, 128, 0, 256 / SP, 500, EPI_STORE, 0, 3, 1, 128, 2, false, false, false, 0, SP>;
    using Up3 = Cfg<PREC, 256, 0, 128, 500, EPI_CONVT, 128, 2, 2, 128, 2, false, false, false, 0, 2>;
    using Dec3 = Cfg<PREC, 128, 128, 128 / SP, 1000, EPI_STORE, 0, is16(PREC) ? 2 : 3, 1, 128, 2, is16(PREC),
                     false, false, 0, SP>;
    using Up2 = Cfg<PREC, 128, 0, 128, 1000, EPI_CONVT, 64, 3, 2, 128, 2>;
    using Dec2Up1 = Cfg<PREC, 64, 64, 64, 2000, EPI_UP, 32, 3, 2, 128, 3, conv_paired(3, PREC), false, true>;
    using Dec1Final = Cfg<PREC, 32, 32, 32, 4000, EPI_FINAL, 0, 3, 1, 96, 4>;
};

// Index of each tensor-core layer in TcNet::w: enc2, enc3, enc4, dec3, dec2, dec1, up3, up2, up1
const int kBlobIndex[9] = {7, 8, 9, 11, 13, 15, 10, 12, 14};

// Host f16 conversion, saturating like the kernels' stores (round to nearest even, +-65504).
__half f16_sat(float x) {
    return __float2half_rn(x > 65504.0f ? 65504.0f : (x < -65504.0f ? -65504.0f : x));
}

struct Packer {
    int prec, es, pw;
    std::vector<unsigned char> bytes;
    size_t put_raw(const void *p, size_t n) {
        size_t off = (bytes.size() + 127) / 128 * 128;
        bytes.resize(off + n);
        std::memcpy(bytes.data() + off, p, n);
        return off;
    }
    void enc(float x, unsigned char *dst) const {
        if (prec == PVF_BF16) {
            __nv_bfloat16 h = __float2bfloat16_rn(x);
            std::memcpy(dst, &h, 2);
        } else if (prec == PVF_FP16) {
            __half h = f16_sat(x);
            std::memcpy(dst, &h, 2);
        } else {
            __nv_fp8_e4m3 q(x);
            std::memcpy(dst, &q, 1);
        }
    }
};

// Per-output-channel fp8 weight scale: amax over the channel / 448.
float fp8_scale(float amax) { return amax > 0.0f ? amax / 448.0f : 1.0f; }

}  // namespace

size_t tc_weight_bytes(int precision, int c0) {
    if (precision == PVF_FP32) return 0;
    // packed weights (< 300 KB; about 1.1 MB for the wide network) + biases + column scales
    return c0 == kC0Max ? 2048 * 1024 : 512 * 1024;
}

bool tc_supported(int precision) { return is16(precision) || precision == PVF_FP8_E4M3; }

// Conv layer W[co][ci][t] -> image [tap][plane][co][PW elements] (6th tap zero when paired).
// ConvT W[ci][co][r] -> image [plane of ci][n = r * CUP + co][PW elements].
bool tc_pack_weights(int precision, const std::vector<LayerF32> &layers, const float *act_scale,
                     std::vector<unsigned char> &out, TcNet *net, unsigned char *dev_base) {
    Packer pk{precision, is16(precision) ? 2 : 1, is16(precision) ? 8 : 16, {}};
    net->precision = precision;
    // the base width from enc2's input channels; the wide network splits enc4 and dec3 into
    // parts (each part's image contiguous) and runs up3 as a ConvT GEMM split by r
    const int c0 = (int)layers[kBlobIndex[0]].shape[1];
    net->c0 = c0;
    const bool wide = c0 == kC0Max;
    const int sp = is16(precision) ? 4 : 2;
    size_t off_w[9], off_b[9], off_s[9];
    for (int li = 0; li < 9; ++li) {
        const LayerF32 &Lw = layers[kBlobIndex[li]];
        const bool up = li >= 6;
        std::vector<unsigned char> img;
        std::vector<float> scale;
        int cout;
        if (!up) {
            cout = (int)Lw.shape[0];
            const int cin = (int)Lw.shape[1];
            const int pin = cin / pk.pw;
            const bool pair = pin == 1;
            const int taps = pair ? 6 : 5;
            scale.assign(cout, 1.0f);
            if (precision == PVF_FP8_E4M3)
                for (int co = 0; co < cout; ++co) {
                    float amax = 0.0f;
                    for (int i = 0; i < cin * 5; ++i) amax = std::max(amax, std::fabs(Lw.w[(size_t)co * cin * 5 + i]));
                    scale[co] = fp8_scale(amax);
                }
            img.assign((size_t)taps * pin * cout * 16, 0);
            for (int t = 0; t < 5; ++t)
                for (int k = 0; k < pin; ++k)
                    for (int co = 0; co < cout; ++co)
                        for (int j = 0; j < pk.pw; ++j) {
                            const int ci = k * pk.pw + j;
                            const float w = Lw.w[((size_t)co * cin + ci) * 5 + t] / scale[co];
                            // paired: group g = t / 2 (N = 2 cout rows for taps 0-3, cout for
                            // tap 4), plane k, row (t % 2) * cout + co; else tap-major planes
                            // wide enc4 / dec3: part co / (cout / sp) of the split; inside the
                            // part tap-major planes of cout / sp rows (enc4, and dec3 in e4m3)
                            // or the paired groups (16-bit dec3)
                            const int cl = cout / sp, cp = co % cl;
                            const size_t row =
                                wide && li == 3 && is16(precision)
                                    ? (size_t)(co / cl) * 5 * pin * cl + (size_t)(t / 2) * pin * 2 * cl +
                                          (size_t)k * (t < 4 ? 2 * cl : cl) + (t % 2) * cl + cp
                                : wide && (li == 2 || li == 3)
                                    ? (size_t)(co / cl) * 5 * pin * cl + ((size_t)t * pin + k) * cl + cp
                                : conv_paired(li, precision) && !(wide && li == 3)
                                    ? (size_t)(t / 2) * pin * 2 * cout + (size_t)k * (t < 4 ? 2 * cout : cout) +
                                          (t % 2) * cout + co
                                    : ((size_t)t * pin + k) * cout + co;
                            pk.enc(w, &img[row * 16 + j * pk.es]);
                        }
        } else {
            const int cin = (int)Lw.shape[0];
            const int cup = (int)Lw.shape[1];
            const int n2 = 2 * cup;
            cout = n2;
            const int p2 = cin / pk.pw;
            scale.assign(n2, 1.0f);
            if (precision == PVF_FP8_E4M3)
                for (int co = 0; co < cup; ++co) {
                    float amax = 0.0f;
                    for (int ci = 0; ci < cin; ++ci)
                        for (int r = 0; r < 2; ++r)
                            amax = std::max(amax, std::fabs(Lw.w[((size_t)ci * cup + co) * 2 + r]));
                    scale[co] = scale[cup + co] = fp8_scale(amax);
                }
            img.assign((size_t)p2 * n2 * 16, 0);
            for (int k = 0; k < p2; ++k)
                for (int n = 0; n < n2; ++n)
                    for (int j = 0; j < pk.pw; ++j) {
                        const int ci = k * pk.pw + j, r = n / cup, co = n % cup;
                        const float w = Lw.w[((size_t)ci * cup + co) * 2 + r] / scale[n];
                        // the wide up3 (a ConvT GEMM split by r): part r's planes of cup rows
                        const size_t row = wide && li == 6 ? (size_t)r * p2 * cup + (size_t)k * cup + co
                                                           : (size_t)k * n2 + n;
                        pk.enc(w, &img[row * 16 + j * pk.es]);
                    }
        }
        off_w[li] = pk.put_raw(img.data(), img.size());
        const size_t nbias = up ? Lw.shape[1] : Lw.shape[0];
        off_b[li] = pk.put_raw(Lw.b, nbias * sizeof(float));
        // fp8 dequantisation scale per accumulator column: input activation scale x weight scale
        std::vector<float> cs(cout, 1.0f);
        if (precision == PVF_FP8_E4M3) {
            // scale of each layer's input tensor
            const int in_idx[9] = {kScaleL1, kScaleL2, kScaleL3, kScaleL3, kScaleL2, kScaleL1,
                                   kScaleE4, kScaleD3, kScaleD2};
            for (int c = 0; c < cout; ++c) cs[c] = act_scale[in_idx[li]] * scale[c];
        }
        off_s[li] = pk.put_raw(cs.data(), cs.size() * sizeof(float));
    }
    // FC images (f16 in the FP16 form, bf16 in the others): element (out o, in i) of layer l at
    // ((i / 8) * R + row) * 16 + (i % 8) * 2 of the layer's image, R rows per plane;
    // row = o for layers 1-5 (R = 32), fc6_row(o) for layer 6 (R = 128)
    std::vector<unsigned char> fcimg(kFcImgBytes, 0);
    for (int l = 0; l < 6; ++l) {
        const LayerF32 &Lw = layers[l];
        const int nout = (int)Lw.shape[0], nin = (int)Lw.shape[1];
        const int rows = l < 5 ? kFcHidden : kFcM6;
        for (int o = 0; o < nout; ++o)
            for (int i = 0; i < nin; ++i) {
                const float wv = Lw.w[(size_t)o * nin + i];
                uint16_t hv;
                if (precision == PVF_FP16) {
                    const __half h = f16_sat(wv);
                    std::memcpy(&hv, &h, 2);
                } else {
                    const __nv_bfloat16 h = __float2bfloat16_rn(wv);
                    std::memcpy(&hv, &h, 2);
                }
                const int row = l < 5 ? o : fc6_row(o);
                std::memcpy(&fcimg[fc_img_off(l) + ((i / 8) * rows + row) * 16 + (i % 8) * 2], &hv, 2);
            }
    }
    const size_t off_fc = pk.put_raw(fcimg.data(), fcimg.size());
    if (pk.bytes.size() > tc_weight_bytes(precision, c0)) return false;
    net->fc_img = dev_base + off_fc;
    for (int li = 0; li < 9; ++li) {
        net->w[li] = dev_base + off_w[li];
        net->b[li] = reinterpret_cast<const float *>(dev_base + off_b[li]);
        net->wscale[li] = reinterpret_cast<const float *>(dev_base + off_s[li]);
    }
    for (int i = 0; i < PVF_N_ACT_SCALES; ++i) net->act_scale[i] = act_scale[i];
    out.swap(pk.bytes);
    return true;
}

template <int PREC, class N>
static cudaError_t run_tc(const TcNet &n, const UnetBuffers &b, int ne, const int32_t *n_dyn, int dyn_base,
                          cudaStream_t s, const ProfHook *prof) {
    const float *sc = n.act_scale;
    auto inv = [&](int i) { return is16(PREC) ? 1.0f : 1.0f / sc[i]; };
    auto cs = [&](int li) { return is16(PREC) ? nullptr : n.wscale[li]; };
    auto W = [&](int li) { return static_cast<const unsigned char *>(n.w[li]); };
    auto U = [](void *p) { return static_cast<unsigned char *>(p); };
    cudaError_t err;
    TcArgs a{};
    a.n_events = ne;
    a.n_dyn = n_dyn;
    a.dyn_base = dyn_base;
    a.status = n.status;
    a.amax = n.amax;
    // one scheduler counter pair per kernel family (each launch leaves it at zero)
    auto sched = [&](int k) { return n.sched + 2 * k; };
    a.sched = sched(0);
    // enc2: p1 (s0) -> e2, p2 (s1)
    a.inA = U(b.s0); a.inB = nullptr; a.out = U(b.e2); a.outp = U(b.s1);
    a.w = W(0); a.bias = n.b[0]; a.cs = cs(0); a.out_inv = inv(kScaleL2); a.amax_out = kScaleL2;
    if ((err = launch_conv<typename N::Enc2>(a, s, prof, "enc2", n.ctas_per_sm[0])) != cudaSuccess) return err;
    // enc3: p2 (s1) -> e3, p3 (s0)
    a.inA = U(b.s1); a.out = U(b.e3); a.outp = U(b.s0); a.sched = sched(1);
    a.w = W(1); a.bias = n.b[1]; a.cs = cs(1); a.out_inv = inv(kScaleL3); a.amax_out = kScaleL3;
    if ((err = launch_conv<typename N::Enc3>(a, s, prof, "enc3", n.ctas_per_sm[1])) != cudaSuccess) return err;
    // enc4 + up3: p3 (s0) -> u3 (up)
    a.inA = U(b.s0); a.out = U(b.up); a.outp = nullptr; a.sched = sched(2);
    a.w = W(2); a.bias = n.b[2]; a.cs = cs(2); a.w2 = W(6); a.bias2 = n.b[6]; a.cs2 = cs(6);
    a.mid_inv = inv(kScaleE4); a.out_inv = inv(kScaleL3); a.amax_mid = kScaleE4; a.amax_out = kScaleL3;
    if ((err = launch_conv<typename N::Enc4Up3>(a, s, prof, "enc4_up3", n.ctas_per_sm[2])) != cudaSuccess) return err;
    // dec3 + up2: [u3 (up), e3] -> u2 (deep)
    a.inA = U(b.up); a.inB = U(b.e3); a.out = U(b.deep); a.sched = sched(3);
    a.w = W(3); a.bias = n.b[3]; a.cs = cs(3); a.w2 = W(7); a.bias2 = n.b[7]; a.cs2 = cs(7);
    a.mid_inv = inv(kScaleD3); a.out_inv = inv(kScaleL2); a.amax_mid = kScaleD3; a.amax_out = kScaleL2;
    if ((err = launch_conv<typename N::Dec3Up2>(a, s, prof, "dec3_up2", n.ctas_per_sm[3])) != cudaSuccess) return err;
    // dec2 + up1: [u2 (deep), e2] -> u1 (up)
    a.inA = U(b.deep); a.inB = U(b.e2); a.out = U(b.up); a.sched = sched(4);
    a.w = W(4); a.bias = n.b[4]; a.cs = cs(4); a.w2 = W(8); a.bias2 = n.b[8]; a.cs2 = cs(8);
    a.mid_inv = inv(kScaleD2); a.out_inv = inv(kScaleL1); a.amax_mid = kScaleD2; a.amax_out = kScaleL1;
    if ((err = launch_conv<typename N::Dec2Up1>(a, s, prof, "dec2_up1", n.ctas_per_sm[4])) != cudaSuccess) return err;
    // dec1 + final conv: [u1 (up), e1] -> logits (float32)
    a.inA = U(b.up); a.inB = U(b.e1); a.out = nullptr; a.w2 = nullptr; a.bias2 = nullptr; a.sched = sched(5);
    a.cs2 = nullptr; a.logits = b.logits; a.final_w = n.final_w; a.amax_out = kScaleD1;
    a.w = W(5); a.bias = n.b[5]; a.cs = cs(5);
    return launch_conv<typename N::Dec1Final>(a, s, prof, "dec1_final", n.ctas_per_sm[5]);
}

// The wide network (base width 32). Activation slots by liveness: e1 | e2 | e3 | deep = e4,
// d3, u1 | up = u3, u2 | s0 = p1, p3 | s1 = p2.
template <int PREC>
static cudaError_t run_tc32(const TcNet &n, const UnetBuffers &b, int ne, const int32_t *n_dyn, int dyn_base,
                            cudaStream_t s, const ProfHook *prof) {
    using N = Net32<PREC>;
    const float *sc = n.act_scale;
    auto inv = [&](int i) { return is16(PREC) ? 1.0f : 1.0f / sc[i]; };
    auto cs = [&](int li) { return is16(PREC) ? nullptr : n.wscale[li]; };
    auto W = [&](int li) { return static_cast<const unsigned char *>(n.w[li]); };
    auto U = [](void *p) { return static_cast<unsigned char *>(p); };
    cudaError_t err;
    TcArgs a{};
    a.n_events = ne;
    a.n_dyn = n_dyn;
    a.dyn_base = dyn_base;
    a.status = n.status;
    a.amax = n.amax;
    auto sched = [&](int k) { return n.sched + 2 * k; };
    // enc2: p1 (s0) -> e2, p2 (s1)
    a.sched = sched(0);
    a.inA = U(b.s0); a.inB = nullptr; a.out = U(b.e2); a.outp = U(b.s1);
    a.w = W(0); a.bias = n.b[0]; a.cs = cs(0); a.out_inv = inv(kScaleL2); a.amax_out = kScaleL2;
    if ((err = launch_conv<typename N::Enc2>(a, s, prof, "enc2", n.ctas_per_sm[0])) != cudaSuccess) return err;
    // enc3: p2 (s1) -> e3, p3 (s0)
    a.inA = U(b.s1); a.out = U(b.e3); a.outp = U(b.s0); a.sched = sched(1);
    a.w = W(1); a.bias = n.b[1]; a.cs = cs(1); a.out_inv = inv(kScaleL3); a.amax_out = kScaleL3;
    if ((err = launch_conv<typename N::Enc3>(a, s, prof, "enc3", n.ctas_per_sm[1])) != cudaSuccess) return err;
    // enc4 (split): p3 (s0) -> e4 (deep)
    a.inA = U(b.s0); a.out = U(b.deep); a.outp = nullptr; a.sched = sched(2);
    a.w = W(2); a.bias = n.b[2]; a.cs = cs(2); a.out_inv = inv(kScaleE4); a.amax_out = kScaleE4;
    if ((err = launch_conv<typename N::Enc4>(a, s, prof, "enc4", n.ctas_per_sm[2])) != cudaSuccess) return err;
    // up3 (ConvT GEMM, split by r): e4 (deep) -> u3 (up)
    a.inA = U(b.deep); a.out = U(b.up);
    a.w = W(6); a.bias = n.b[6]; a.cs = cs(6); a.out_inv = inv(kScaleL3); a.amax_out = kScaleL3;
    if ((err = launch_conv<typename N::Up3>(a, s, prof, "up3", n.ctas_per_sm[2])) != cudaSuccess) return err;
    // dec3 (split): [u3 (up), e3] -> d3 (deep)
    a.inA = U(b.up); a.inB = U(b.e3); a.out = U(b.deep); a.sched = sched(3);
    a.w = W(3); a.bias = n.b[3]; a.cs = cs(3); a.out_inv = inv(kScaleD3); a.amax_out = kScaleD3;
    if ((err = launch_conv<typename N::Dec3>(a, s, prof, "dec3", n.ctas_per_sm[3])) != cudaSuccess) return err;
    // up2 (ConvT GEMM): d3 (deep) -> u2 (up)
    a.inA = U(b.deep); a.inB = nullptr; a.out = U(b.up);
    a.w = W(7); a.bias = n.b[7]; a.cs = cs(7); a.out_inv = inv(kScaleL2); a.amax_out = kScaleL2;
    if ((err = launch_conv<typename N::Up2>(a, s, prof, "up2", n.ctas_per_sm[3])) != cudaSuccess) return err;
    // dec2 + up1: [u2 (up), e2] -> u1 (deep)
    a.inA = U(b.up); a.inB = U(b.e2); a.out = U(b.deep); a.sched = sched(4);
    a.w = W(4); a.bias = n.b[4]; a.cs = cs(4); a.w2 = W(8); a.bias2 = n.b[8]; a.cs2 = cs(8);
    a.mid_inv = inv(kScaleD2); a.out_inv = inv(kScaleL1); a.amax_mid = kScaleD2; a.amax_out = kScaleL1;
    if ((err = launch_conv<typename N::Dec2Up1>(a, s, prof, "dec2_up1", n.ctas_per_sm[4])) != cudaSuccess)
        return err;
    // dec1 + final conv: [u1 (deep), e1] -> logits (float32)
    a.inA = U(b.deep); a.inB = U(b.e1); a.out = nullptr; a.w2 = nullptr; a.bias2 = nullptr; a.sched = sched(5);
    a.cs2 = nullptr; a.logits = b.logits; a.final_w = n.final_w; a.amax_out = kScaleD1;
    a.w = W(5); a.bias = n.b[5]; a.cs = cs(5);
    return launch_conv<typename N::Dec1Final>(a, s, prof, "dec1_final", n.ctas_per_sm[5]);
}

// The enc2 kernel alone with its MMA thread stalled for stall_us (tests of the bounded waits).
template <int PREC>
static cudaError_t stall_tc(const TcNet &n, const UnetBuffers &b, int ne, uint32_t stall_us, cudaStream_t s) {
    using N = Net<PREC>;
    TcArgs a{};
    a.n_events = ne;
    a.status = n.status;
    a.sched = n.sched;
    a.inA = static_cast<const unsigned char *>(b.s0);
    a.out = static_cast<unsigned char *>(b.e2);
    a.outp = static_cast<unsigned char *>(b.s1);
    a.w = static_cast<const unsigned char *>(n.w[0]);
    a.bias = n.b[0];
    a.cs = is16(PREC) ? nullptr : n.wscale[0];
    a.out_inv = is16(PREC) ? 1.0f : 1.0f / n.act_scale[kScaleL2];
    a.stall_test_us = stall_us;
    return launch_conv<typename N::Enc2>(a, s, nullptr, "enc2", n.ctas_per_sm[0]);
}

cudaError_t launch_stall_test_tc(const TcNet &net, const UnetBuffers &b, int n, uint32_t stall_us,
                                 cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    switch (net.precision) {
    case PVF_BF16: return stall_tc<PVF_BF16>(net, b, n, stall_us, s);
    case PVF_FP16: return stall_tc<PVF_FP16>(net, b, n, stall_us, s);
    case PVF_FP8_E4M3: return stall_tc<PVF_FP8_E4M3>(net, b, n, stall_us, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_unet_tc(const TcNet &net, const UnetBuffers &b, int n, const int32_t *n_dyn, int dyn_base,
                           cudaStream_t s, const ProfHook *prof) {
    if (n <= 0) return cudaSuccess;
    if (net.c0 == kC0Max) {
        switch (net.precision) {
        case PVF_BF16: return run_tc32<PVF_BF16>(net, b, n, n_dyn, dyn_base, s, prof);
        case PVF_FP16: return run_tc32<PVF_FP16>(net, b, n, n_dyn, dyn_base, s, prof);
        case PVF_FP8_E4M3: return run_tc32<PVF_FP8_E4M3>(net, b, n, n_dyn, dyn_base, s, prof);
        default: return cudaErrorInvalidValue;
        }
    }
    if (net.iv) {
        switch (net.precision) {
        case PVF_BF16: return run_tc<PVF_BF16, NetIv<PVF_BF16>>(net, b, n, n_dyn, dyn_base, s, prof);
        case PVF_FP16: return run_tc<PVF_FP16, NetIv<PVF_FP16>>(net, b, n, n_dyn, dyn_base, s, prof);
        case PVF_FP8_E4M3: return run_tc<PVF_FP8_E4M3, NetIv<PVF_FP8_E4M3>>(net, b, n, n_dyn, dyn_base, s, prof);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (net.precision) {
    case PVF_BF16: return run_tc<PVF_BF16, Net<PVF_BF16>>(net, b, n, n_dyn, dyn_base, s, prof);
    case PVF_FP16: return run_tc<PVF_FP16, Net<PVF_FP16>>(net, b, n, n_dyn, dyn_base, s, prof);
    case PVF_FP8_E4M3: return run_tc<PVF_FP8_E4M3, Net<PVF_FP8_E4M3>>(net, b, n, n_dyn, dyn_base, s, prof);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pvf
