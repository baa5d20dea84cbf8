// Mixed-precision coagulation step on the 5th-generation tensor cores.
//
// The gain/loss redistribution of Eq. (smol) is a contraction over pairs:
//   d rho_k / dt = S^2 sum_q Bt[k][q] A[c][q],
// with S = sum_k |rho_k| per cell, x = rho / S, and per pair p = (i, j <= i)
// two columns q: A = x_i x_j K_ij p_coag,ij and A = x_i x_j K_ij p_frag,ij.
// Bt holds the fixed net redistribution coefficients per unit n_i n_j K and
// outcome: coagulation into the two bins of Eq. Cijk minus the two colliding
// grains, and remnant into those of Eq. Rijk plus fragments by N_k of
// Eq. Nijk minus the two colliding grains (1/2 at i = j), divided by m_i m_j.
// It is built once on the host in double-double.  Carrying p_coag and p_frag
// each in its own column keeps both accurate in FP32 whichever dominates.
//
// Layout on chip (one CTA per SM, persistent over all right-hand sides):
//   MMA M = 128 bins (Bt, streamed as swizzled 32 KB TF32 hi/lo tiles by the
//   bulk-copy engine), MMA N = NS cell slots (generated operand), K = 32
//   TF32 elements (16 pairs) per block.  Each block issues the four products
//   of (Bt_hi + Bt_lo)(A_hi + A_lo), hi and lo rounded to nearest TF32: hi x
//   hi into one of several FP32 accumulators [128 lanes x NS columns] in TMEM
//   (a contiguous share of the blocks each), the three corrections into one
//   more; the epilogue adds them with a compensated (Neumaier) FP32 sum.
// Warp roles: warp 0 bulk-copy producer, warp 1 MMA issuer and TMEM owner,
// warps 2..9 generate A (x_i x_j K split into hi/lo in the SW128 K-major
// layout) and, between right-hand sides, run the per-slot FP64 logic: the
// mass budget (sum_k f_k = 0 restored in FP64), the Bogacki-Shampine 3(2)
// stages, the error norm, step control and refilling a slot with the next
// cell when one finishes.
//
// Every mbarrier wait is bounded by a clock limit; a wait that runs out
// records an error code in the status word and the kernel winds down.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "coag_internal.h"

namespace cdc {
namespace {

constexpr int kGenWarps = 8;
constexpr int kMaxMain = 8;                       // TMEM accumulators for the hi x hi products
constexpr int kCStages = 4;                       // generated-tile ring depth
constexpr int kMaxSB = 8;                         // mapping-tile ring depth, at most
constexpr int kThreads = 64 + 32 * kGenWarps;
constexpr int kTileBytes = kMBins * 128;          // one 128-row x 128 B TF32 tile
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz
constexpr double A21 = 0.5, A32 = 0.75;
constexpr double B1 = 2.0 / 9.0, B2 = 1.0 / 3.0, B3 = 4.0 / 9.0;
constexpr double E1 = -5.0 / 72.0, E2 = 1.0 / 12.0, E3 = 1.0 / 9.0, E4 = -1.0 / 8.0;

// Bytes of one pipeline stage: Bt hi/lo tiles and the generated hi/lo tiles,
// rounded up to keep every stage 1024-byte aligned.
__host__ __device__ constexpr int stage_size(int NS)
{
    return ((2 * kTileBytes + 2 * NS * 128 + 1023) / 1024) * 1024;
}

enum Mode { MODE_STEP = 0, MODE_RHS = 1, MODE_REPLAY = 2 };
enum ErrCode { ERR_WAIT_PRODUCER = 1, ERR_WAIT_MMA = 2, ERR_WAIT_GEN = 3, ERR_WAIT_EPI = 4 };

struct MixedArgs {
    DevTables t;
    const float2 *K32;          // [n_cells][n_blk*16]
    double *rho;                // state in/out (STEP, REPLAY) or input (RHS)
    double *drho;               // output (RHS)
    double t_span;
    double *dt_cell;
    double rtol, atol_rel;
    long long max_steps;
    const double *replay_h;
    const long long *replay_n;
    long long replay_stride;
    CellOut *out;
    int *err;                   // device status word
    int *queue;                 // global work-queue head (cells past the initial fill)
    double *work;               // [grid][NS][5][N] FP64 slot state
    double *rec_dt;
    long long rec_cap;
    long long *rec_n;
    int *rec_status;
    int NS, S, XS, mode;
    int SB, NB8;                // mapping-tile ring depth, tile rows copied (bins rounded to 8)
};

struct __align__(16) Slot {
    double t, h, hs, S, Sx, atol;
    long long nacc, nrej, nrep;
    int cell, phase, last, status;
};

// ---- PTX wrappers ----------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(su32(b)), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait: false when the clock limit runs out or another role failed.
__device__ __noinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *s_err, int code)
{
    const long long t0 = clock64();
    for (int it = 0;; ++it) {
        if (mbar_test(b, parity)) return true;
        if ((it & 63) == 63) {
            if (*s_err) return false;
            if (clock64() - t0 > kWaitCycles) { atomicCAS((int *)s_err, 0, code); return false; }
        }
    }
}
// The same wait, with one answer for the whole warp (all 32 lanes call it).
__device__ __forceinline__ bool wwait(uint64_t *b, uint32_t parity, volatile int *s_err, int code)
{
    // fast path: the phase is usually complete already
    if (__all_sync(0xffffffffu, mbar_test(b, parity))) return true;
    return __all_sync(0xffffffffu, mbar_wait(b, parity, s_err, code));
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(su32(dst)), "l"(src), "r"(bytes), "r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: 8-row groups
// 1024 B apart (SBO), descriptor version 1, layout code 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// Instruction descriptor, kind::tf32: D F32, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(dt), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 8; q++) v[q] = __uint_as_float(r[q]);
}
// Generator-group barrier on an mbarrier (256 arrivals), with a bounded wait
// so that a group member that gave up cannot hang the others.
__device__ __forceinline__ bool gen_sync(uint64_t *gbar, uint32_t &phase, volatile int *s_err)
{
    mbar_arrive(gbar);
    const bool ok = wwait(gbar, phase & 1, s_err, ERR_WAIT_EPI);
    phase++;
    return ok;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// TF32 split, both parts rounded to nearest: hi = rn_tf32(v), lo =
// rn_tf32(v - hi).  The tensor core then sees exact TF32 values and
// hi + lo matches v to 2^-22 relative, without the bias of truncation.
__device__ __forceinline__ float tf32_rn(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// ---- per-slot logic (one warp per slot, lanes over bins) ------------------

// Slot state in global scratch (per slot 5 N doubles are reserved): the state
// y in FP64, its scaled copy yx = y / Sx and the stage right-hand sides in the
// same scaled units (kx = f / Sx = Sx D) in FP32.  The stage inputs, the error
// norm and the step controller work in FP32 (their rounding sits below the
// contraction's own ~3e-7); FP64 holds the state and the mass budget of every
// accepted increment, so total mass is conserved to FP64 rounding.
struct SlotBufs { double *y; float *yx, *k1, *k2, *k3; };

__device__ __forceinline__ SlotBufs slot_bufs(const MixedArgs &a, int slot)
{
    const int N = a.t.N;
    double *base = a.work + ((size_t)blockIdx.x * a.NS + slot) * 5 * (size_t)N;
    float *f = (float *)(base + N);
    return {base, f, f + N, f + 2 * N, f + 3 * N};
}

// Load cell c into slot: state, scales, phase 0 (or mark the slot empty).
__device__ void slot_load(const MixedArgs &a, Slot &sl, float *xrow, int slot, int c)
{
    const int N = a.t.N, lane = threadIdx.x & 31;
    if (c < 0) {
        for (int k = lane; k < a.XS; k += 32) xrow[k] = 0.f;
        if (lane == 0) sl.cell = -1;
        return;
    }
    SlotBufs B = slot_bufs(a, slot);
    const double *rc = a.rho + (size_t)c * N;
    double s = 0.0, sa = 0.0;
    for (int k = lane; k < N; k += 32) {
        const double v = rc[k];
        B.y[k] = v;
        s += v;
        sa += fabs(v);
    }
    s = warp_sum(s);
    sa = warp_sum(sa);
    const double Sx = sa > 0.0 ? sa : 1.0;
    const double r = 1.0 / Sx;
    for (int k = lane; k < a.XS; k += 32) {
        const float v = (k < N) ? (float)(B.y[k] * r) : 0.f;
        if (k < N) B.yx[k] = v;
        xrow[k] = v;
    }
    if (lane == 0) {
        sl.cell = c;
        sl.phase = 0;
        sl.S = s;
        sl.Sx = Sx;
        sl.atol = a.atol_rel * s;
        sl.t = 0.0;
        sl.h = (a.mode == MODE_STEP && a.dt_cell) ? a.dt_cell[c] : 0.0;
        sl.hs = 0.0;
        sl.nacc = sl.nrej = sl.nrep = 0;
        sl.last = 0;
        sl.status = CUDISC_OK;
    }
}

__device__ void slot_finish(const MixedArgs &a, Slot &sl, int slot)
{
    const int N = a.t.N, lane = threadIdx.x & 31;
    const int c = sl.cell;
    if (a.mode != MODE_RHS) {
        SlotBufs B = slot_bufs(a, slot);
        double *rc = a.rho + (size_t)c * N;
        double s1 = 0.0;
        for (int k = lane; k < N; k += 32) { rc[k] = B.y[k]; s1 += B.y[k]; }
        s1 = warp_sum(s1);
        if (lane == 0) {
            CellOut o;
            o.n_acc = sl.nacc; o.n_rej = sl.nrej; o.h_last = sl.h;
            o.mass_err = sl.S > 0.0 ? fabs(s1 / sl.S - 1.0) : 0.0;
            o.status = sl.status; o.pad = 0;
            a.out[c] = o;
            if (a.dt_cell && a.mode == MODE_STEP) a.dt_cell[c] = sl.h;
            if (a.rec_n) a.rec_n[c] = sl.nacc;
            if (a.rec_status) a.rec_status[c] = sl.status;
        }
    }
}

// Accept an increment dx (scaled units, FP32) into the FP64 state: the
// residual of sum_k dx_k is moved in proportion to |dx_k| (mass budget),
// then y += Sx dx and yx = y / Sx.
__device__ void commit_increment(const Slot &sl, SlotBufs B, int N, const float *dx)
{
    const int lane = threadIdx.x & 31;
    double d[(kMBins + 31) / 32];
    double s = 0.0, sa = 0.0;
#pragma unroll
    for (int m = 0; m < (kMBins + 31) / 32; m++) {
        const int k = lane + 32 * m;
        d[m] = (k < N) ? (double)dx[m] * sl.Sx : 0.0;
        s += d[m];
        sa += fabs(d[m]);
    }
    s = warp_sum(s);
    sa = warp_sum(sa);
    const double q = sa > 0.0 ? s / sa : 0.0;
    const double r = 1.0 / sl.Sx;
#pragma unroll
    for (int m = 0; m < (kMBins + 31) / 32; m++) {
        const int k = lane + 32 * m;
        if (k < N) {
            const double y = B.y[k] + (d[m] - q * fabs(d[m]));
            B.y[k] = y;
            B.yx[k] = (float)(y * r);
        }
    }
    __syncwarp();
}

// First stage input x = yx + hs A21 k1 after choosing the step (shared by
// the first step and every step after an accept or reject).
__device__ bool begin_step(const MixedArgs &a, Slot &sl, float *xrow, SlotBufs B)
{
    const int N = a.t.N, lane = threadIdx.x & 31;
    if (sl.nacc + sl.nrej >= a.max_steps) { sl.status = CUDISC_EMAXSTEPS; return false; }
    sl.last = (sl.h >= a.t_span - sl.t);
    sl.hs = sl.last ? (a.t_span - sl.t) : sl.h;
    const float c1 = (float)(sl.hs * A21);
    for (int k = lane; k < N; k += 32) xrow[k] = B.yx[k] + c1 * B.k1[k];
    sl.phase = 1;
    return true;
}

// Process one right-hand side result, D = sum of the TMEM accumulators for
// this slot (kx = Sx D in scaled units).  Returns true when the slot
// finished its cell.
__device__ bool slot_advance(const MixedArgs &a, Slot &sl, float *xrow, const float *Drow, int slot)
{
    const int N = a.t.N, lane = threadIdx.x & 31;
    constexpr int MB = (kMBins + 31) / 32;
    SlotBufs B = slot_bufs(a, slot);
    const float sx = (float)sl.Sx;
    float kv[MB];
#pragma unroll
    for (int m = 0; m < MB; m++) {
        const int k = lane + 32 * m;
        kv[m] = (k < N) ? sx * Drow[k] : 0.f;
    }
    if (a.mode == MODE_RHS) {
        // d rho / dt = Sx^2 D with the FP64 mass budget
        double fv[MB], s = 0.0, sa = 0.0;
#pragma unroll
        for (int m = 0; m < MB; m++) {
            const int k = lane + 32 * m;
            fv[m] = (k < N) ? sl.Sx * sl.Sx * (double)Drow[k] : 0.0;
            s += fv[m];
            sa += fabs(fv[m]);
        }
        s = warp_sum(s);
        sa = warp_sum(sa);
        const double q = sa > 0.0 ? s / sa : 0.0;
#pragma unroll
        for (int m = 0; m < MB; m++) {
            const int k = lane + 32 * m;
            if (k < N) a.drho[(size_t)sl.cell * N + k] = fv[m] - q * fabs(fv[m]);
        }
        return true;
    }
    float *dst = sl.phase == 0 ? B.k1 : sl.phase == 1 ? B.k2 : sl.phase == 2 ? B.k3 : nullptr;
    if (dst) {
#pragma unroll
        for (int m = 0; m < MB; m++) {
            const int k = lane + 32 * m;
            if (k < N) dst[k] = kv[m];
        }
        __syncwarp();
    }
    if (a.mode == MODE_REPLAY) {
        const long long nh = a.replay_n[sl.cell];
        const double hh = nh > 0 ? a.replay_h[(size_t)sl.cell * a.replay_stride + sl.nrep] : 0.0;
        if (sl.phase == 0) {
            if (nh == 0) return true;
            const float c1 = (float)(hh * A21);
            for (int k = lane; k < N; k += 32) xrow[k] = B.yx[k] + c1 * B.k1[k];
            sl.phase = 1;
        } else if (sl.phase == 1) {
            const float c2 = (float)(hh * A32);
            for (int k = lane; k < N; k += 32) xrow[k] = B.yx[k] + c2 * B.k2[k];
            sl.phase = 2;
        } else {
            const float b1 = (float)(hh * B1), b2 = (float)(hh * B2), b3 = (float)(hh * B3);
            float dx[MB];
#pragma unroll
            for (int m = 0; m < MB; m++) {
                const int k = lane + 32 * m;
                dx[m] = (k < N) ? b1 * B.k1[k] + b2 * B.k2[k] + b3 * B.k3[k] : 0.f;
            }
            commit_increment(sl, B, N, dx);
            sl.nrep++;
            sl.nacc = sl.nrep;
            if (sl.nrep >= nh) return true;
            for (int k = lane; k < N; k += 32) xrow[k] = B.yx[k];
            sl.phase = 0;
        }
        return false;
    }
    // adaptive Bogacki-Shampine 3(2)
    switch (sl.phase) {
    case 0: {
        if (!(sl.h > 0.0)) {
            const float atolx = (float)(sl.atol / sl.Sx);
            float q = INFINITY;
            for (int k = lane; k < N; k += 32)
                if (B.k1[k] != 0.f) q = fminf(q, (fabsf(B.yx[k]) + atolx) / fabsf(B.k1[k]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) q = fminf(q, __shfl_xor_sync(0xffffffffu, q, o));
            sl.h = isfinite(q) ? 0.1 * (double)q : a.t_span;
            if (sl.h > a.t_span) sl.h = a.t_span;
        }
        return !begin_step(a, sl, xrow, B);
    }
    case 1: {
        const float c2 = (float)(sl.hs * A32);
        for (int k = lane; k < N; k += 32) xrow[k] = B.yx[k] + c2 * B.k2[k];
        sl.phase = 2;
        return false;
    }
    case 2: {
        const float b1 = (float)(sl.hs * B1), b2 = (float)(sl.hs * B2), b3 = (float)(sl.hs * B3);
        for (int k = lane; k < N; k += 32)
            xrow[k] = B.yx[k] + (b1 * B.k1[k] + b2 * B.k2[k] + b3 * B.k3[k]);
        sl.phase = 3;
        return false;
    }
    default: {
        // phase 3: kv holds k4 = f(y1); y1 = yx + dx is the stage input
        const float b1 = (float)(sl.hs * B1), b2 = (float)(sl.hs * B2), b3 = (float)(sl.hs * B3);
        const float e1 = (float)(sl.hs * E1), e2 = (float)(sl.hs * E2), e3 = (float)(sl.hs * E3),
                    e4 = (float)(sl.hs * E4);
        const float atolx = (float)(sl.atol / sl.Sx), rtol = (float)a.rtol;
        float dx[MB];
        float E = 0.f, ymin = INFINITY, fin = 1.f;
#pragma unroll
        for (int m = 0; m < MB; m++) {
            const int k = lane + 32 * m;
            dx[m] = 0.f;
            if (k < N) {
                const float k1 = B.k1[k], k2 = B.k2[k], k3 = B.k3[k], yx = B.yx[k];
                dx[m] = b1 * k1 + b2 * k2 + b3 * k3;
                const float y1 = yx + dx[m];
                const float e = e1 * k1 + e2 * k2 + e3 * k3 + e4 * kv[m];
                const float sc = atolx + rtol * fmaxf(fabsf(yx), fabsf(y1));
                const float r = fabsf(e) / sc;
                if (!isfinite(r) || !isfinite(y1)) fin = 0.f;
                if (r > E) E = r;
                if (y1 < ymin) ymin = y1;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            E = fmaxf(E, __shfl_xor_sync(0xffffffffu, E, o));
            ymin = fminf(ymin, __shfl_xor_sync(0xffffffffu, ymin, o));
            fin = fminf(fin, __shfl_xor_sync(0xffffffffu, fin, o));
        }
        const bool finite = fin > 0.5f;
        if (finite && E <= 1.f && ymin >= -atolx) {
            commit_increment(sl, B, N, dx);
            sl.t = sl.last ? a.t_span : sl.t + sl.hs;
#pragma unroll
            for (int m = 0; m < MB; m++) {
                const int k = lane + 32 * m;
                if (k < N) B.k1[k] = kv[m];                 // FSAL
            }
            __syncwarp();
            if (lane == 0 && a.rec_dt && sl.nacc < a.rec_cap)
                a.rec_dt[(size_t)sl.cell * a.rec_cap + sl.nacc] = sl.hs;
            sl.nacc++;
            double fac = (E > 0.f) ? 0.9 * pow((double)E, -1.0 / 3.0) : 5.0;
            fac = fmin(fmax(fac, 0.2), 5.0);
            if (!(sl.last && sl.hs < sl.h)) sl.h = sl.hs * fac;
            if (sl.t >= a.t_span) return true;
        } else {
            sl.nrej++;
            double fac;
            if (!finite) fac = 0.2;
            else if (E > 1.f) fac = fmax(0.9 * pow((double)E, -1.0 / 3.0), 0.2);
            else fac = 0.5;
            sl.h = sl.hs * fac;
            if (sl.h < 1e-14 * a.t_span) { sl.status = finite ? CUDISC_EDTMIN : CUDISC_ENONFINITE; return true; }
        }
        return !begin_step(a, sl, xrow, B);
    }
    }
}

// Generate one thread's share (P pairs of one cell row) of a block's operand
// tile: a = x_i x_j K, b = x_i x_j K p_frag, each split into TF32 hi and lo
// and stored at its place in the SW128 K-major tiles.  K comes from the
// stage's staged rows (bulk-copied by the producer), x from the slot's row.
template <int P>
struct KRegs { float v[2 * P]; };

// Load one thread's K share of block b (P pairs, {K, K p_frag} each).
template <int P>
__device__ __forceinline__ void load_k(KRegs<P> &k, const float2 *kbase, int b)
{
    const float *src = (const float *)(kbase + (size_t)b * kBlkPairs);
    if constexpr (P == 4) {
        const float4 a0 = __ldg((const float4 *)src), a1 = __ldg((const float4 *)src + 1);
        k.v[0] = a0.x; k.v[1] = a0.y; k.v[2] = a0.z; k.v[3] = a0.w;
        k.v[4] = a1.x; k.v[5] = a1.y; k.v[6] = a1.z; k.v[7] = a1.w;
    } else if constexpr (P == 2) {
        const float4 a0 = __ldg((const float4 *)src);
        k.v[0] = a0.x; k.v[1] = a0.y; k.v[2] = a0.z; k.v[3] = a0.w;
    } else {
        const float2 a0 = __ldg((const float2 *)src);
        k.v[0] = a0.x; k.v[1] = a0.y;
    }
}

template <int P>
__device__ __forceinline__ void gen_block(float *chi, float *clo, const KRegs<P> &kr, const float *xr,
                                          int bi, int bj0, int t0, int row, bool active)
{
    float va[2 * P];
    if (active) {
        const float xi = xr[bi];
        float xj[P];
        const float *kv = kr.v;
        if constexpr (P == 4) {
            const float4 v = *(const float4 *)(xr + bj0 + t0);
            xj[0] = v.x; xj[1] = v.y; xj[2] = v.z; xj[3] = v.w;
        } else if constexpr (P == 2) {
            const float2 v = *(const float2 *)(xr + bj0 + t0);
            xj[0] = v.x; xj[1] = v.y;
        } else {
            xj[0] = xr[bj0 + t0];
        }
#pragma unroll
        for (int u = 0; u < P; u++) {
            const float xx = xi * xj[u];
            va[2 * u] = xx * kv[2 * u];
            va[2 * u + 1] = xx * kv[2 * u + 1];
        }
    } else {
#pragma unroll
        for (int u = 0; u < 2 * P; u++) va[u] = 0.f;
    }
    float vh[2 * P], vl[2 * P];
#pragma unroll
    for (int u = 0; u < 2 * P; u++) {
        vh[u] = tf32_rn(va[u]);
        vl[u] = tf32_rn(va[u] - vh[u]);
    }
    const int e0 = 2 * t0;                                // first element of the share
#pragma unroll
    for (int q = 0; q < (2 * P + 3) / 4; q++) {
        const int e = e0 + 4 * q;
        const int off = row * 32 + ((((e >> 2) ^ (row & 7)) << 2) | (e & 3));
        if constexpr (P >= 2) {
            *(float4 *)(chi + off) = make_float4(vh[4 * q], vh[4 * q + 1], vh[4 * q + 2], vh[4 * q + 3]);
            *(float4 *)(clo + off) = make_float4(vl[4 * q], vl[4 * q + 1], vl[4 * q + 2], vl[4 * q + 3]);
        } else {
            *(float2 *)(chi + off) = make_float2(vh[0], vh[1]);
            *(float2 *)(clo + off) = make_float2(vl[0], vl[1]);
        }
    }
}

// One pass of a generator thread over all blocks: K loads run two blocks
// ahead in registers; a row without a cell writes its zeros once per stage
// in the pass and is skipped afterwards.
template <int P>
__device__ __forceinline__ bool gen_pass(const MixedArgs &a, uint8_t *cring, int cstride,
                                         const float2 *kbase, const float *xr, uint64_t *c_empty,
                                         uint64_t *c_full, volatile int *s_err, long long g0, int n_blk,
                                         int SC, int NS, int row, int t0, bool active, int lane)
{
    KRegs<P> k0, k1, k2;
    if (active) {
        load_k<P>(k0, kbase, 0);
        if (n_blk > 1) load_k<P>(k1, kbase, 1);
    }
    long long g = g0;
    int s = (int)(g0 % SC);
    uint32_t u = (uint32_t)(g0 / SC);
    for (int b = 0; b < n_blk; b++, g++) {
        if (active && b + 2 < n_blk) load_k<P>(k2, kbase, b + 2);
        if (g >= SC && !wwait(&c_empty[s], (u + 1) & 1, s_err, ERR_WAIT_GEN)) return false;
        if (active || b < SC) {
            float *chi = (float *)(cring + (size_t)s * cstride);
            float *clo = chi + NS * 32;
            const int bi = __ldg(a.t.blk_i + b), bj0 = __ldg(a.t.blk_j0 + b);
            gen_block<P>(chi, clo, k0, xr, bi, bj0, t0, row, active);
            fence_async_smem();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&c_full[s]);
        if (++s == SC) { s = 0; u++; }
        k0 = k1;
        k1 = k2;
    }
    return true;
}

// ---- the kernel --------------------------------------------------------------

__global__ void __launch_bounds__(kThreads, 1) step_mixed_kernel(MixedArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int NS = a.NS, XS = a.XS, N = a.t.N, n_blk = a.t.n_blk;
    const int SB = a.SB, SC = kCStages;
    const int half_bytes = a.NB8 * 128;                 // rows of one Bt tile copied
    const int bstride = 2 * half_bytes;                 // hi then lo, both 1024-aligned
    const int cstride = 2 * NS * 128;
    uint8_t *bring = sm;                                // mapping tiles (also the D staging area)
    uint8_t *cring = bring + (size_t)SB * bstride;      // generated tiles
    float *xrows = (float *)(cring + (size_t)SC * cstride);
    Slot *slots = (Slot *)(xrows + (size_t)NS * XS);
    uint64_t *bars = (uint64_t *)(slots + NS);
    uint64_t *bt_full = bars, *bt_empty = bars + SB;
    uint64_t *c_full = bars + 2 * SB, *c_empty = bars + 2 * SB + SC;
    uint64_t *done = bars + 2 * SB + 2 * SC, *go = done + 1, *gbar = done + 2, *fin = done + 3;
    __shared__ uint32_t s_tmem;
    __shared__ int s_err, s_continue;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // TMEM: nacc accumulators for the hi x hi products, each taking a
    // contiguous share of the blocks (every one gets at least one), plus one
    // for the three 2^-11-smaller correction products of every block.  FP32
    // accumulation error grows with the additions per accumulator; the
    // epilogue adds them with a compensated (Neumaier) FP32 sum.
    int nmain = 512 / NS - 1;
    if (nmain > kMaxMain) nmain = kMaxMain;
    const int nacc = n_blk < nmain ? n_blk : nmain;
    const int tcols = (nacc + 1) * NS;
    const uint32_t ncols = tcols <= 32 ? 32 : tcols <= 64 ? 64 : tcols <= 128 ? 128 : tcols <= 256 ? 256 : 512;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SB; s++) {
            mbar_init(&bt_full[s], 1);
            mbar_init(&bt_empty[s], 1);
        }
        for (int s = 0; s < SC; s++) {
            mbar_init(&c_full[s], kGenWarps);
            mbar_init(&c_empty[s], 1);
        }
        mbar_init(done, 1);
        mbar_init(go, 1);
        mbar_init(gbar, 32 * kGenWarps);
        mbar_init(fin, 1);
        s_err = 0;
        s_continue = 1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(&s_tmem)), "r"(ncols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // initial slot fill: slot s takes cell blockIdx.x + s * gridDim.x
    if (warp >= 2) {
        for (int s = warp - 2; s < NS; s += kGenWarps) {
            const int c = blockIdx.x + s * gridDim.x;
            slot_load(a, slots[s], xrows + (size_t)s * XS, s, c < a.t.n_cells ? c : -1);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        // ---- producer: mapping tiles (rows 0..NB8-1 of hi and lo) by the bulk-copy engine ----
        long long g = 0;
        int ps = 0;
        uint32_t pu = 0;
        for (int r = 0;; r++) {
            if (r > 0) {
                if (!wwait(go, (r - 1) & 1, &s_err, ERR_WAIT_PRODUCER)) break;
                if (!s_continue) break;
            }
            bool ok = true;
            for (int b = 0; b < n_blk; b++, g++) {
                const int s = ps;
                const uint32_t u = pu;
                if (++ps == SB) { ps = 0; pu++; }      // ring position without divisions
                if (g >= SB && !wwait(&bt_empty[s], (u + 1) & 1, &s_err, ERR_WAIT_PRODUCER)) { ok = false; break; }
                if (lane == 0) {
                    uint8_t *dst = bring + (size_t)s * bstride;
                    const uint8_t *src = (const uint8_t *)(a.t.Btiles + (size_t)b * (2 * kTileBytes / 16));
                    mbar_expect_tx(&bt_full[s], 2 * half_bytes);
                    bulk_g2s(dst, src, half_bytes, &bt_full[s]);
                    bulk_g2s(dst + half_bytes, src + kTileBytes, half_bytes, &bt_full[s]);
                }
                __syncwarp();
            }
            if (!ok) break;
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        const uint32_t idesc = idesc_tf32(kMBins, NS);
        long long g = 0;
        int ms = 0, mc = 0;
        uint32_t mu = 0, mv = 0;
        for (int r = 0;; r++) {
            if (r > 0) {
                if (!wwait(go, (r - 1) & 1, &s_err, ERR_WAIT_MMA)) break;
                if (!s_continue) break;
            }
            bool ok = true;
            int ch = 0, ch_next = (n_blk + nacc - 1) / nacc;   // hi x hi accumulator of the block
            bool first = true;
            for (int b = 0; b < n_blk; b++, g++) {
                const int sb = ms, sc = mc;
                const uint32_t ub = mu, uc = mv;
                if (++ms == SB) { ms = 0; mu++; }
                if (++mc == SC) { mc = 0; mv++; }
                if (b == ch_next) { ch++; ch_next = (int)(((long long)(ch + 1) * n_blk + nacc - 1) / nacc); first = true; }
                if (!wwait(&bt_full[sb], ub & 1, &s_err, ERR_WAIT_MMA) ||
                    !wwait(&c_full[sc], uc & 1, &s_err, ERR_WAIT_MMA)) { ok = false; break; }
                tc_fence_after();
                if (lane == 0) {
                    const uint32_t bt_hi = su32(bring + (size_t)sb * bstride), bt_lo = bt_hi + half_bytes;
                    const uint32_t c_hi = su32(cring + (size_t)sc * cstride), c_lo = c_hi + NS * 128;
                    const uint64_t dbh = sw128_desc(bt_hi), dbl = sw128_desc(bt_lo);
                    const uint64_t dch = sw128_desc(c_hi), dcl = sw128_desc(c_lo);
                    // the pass over all blocks is split across nacc TMEM
                    // accumulators (contiguous block ranges) summed later in FP64
                    const uint32_t dt = tmem + (uint32_t)(ch * NS);
                    const uint32_t dc = tmem + (uint32_t)(nacc * NS);
                    // hi x hi into the block's accumulator; hi x lo, lo x hi and
                    // lo x lo into the correction accumulator
                    mma_tf32(dt, dbh, dch, idesc, first ? 0u : 1u);
                    mma_tf32(dc, dbh, dcl, idesc, b > 0 ? 1u : 0u);
                    mma_tf32(dc, dbl, dch, idesc, 1u);
                    mma_tf32(dc, dbl, dcl, idesc, 1u);
#pragma unroll
                    for (int kk = 1; kk < 4; kk++) {
                        const uint64_t adv = (uint64_t)(kk * 2);   // 32 bytes per K step
                        mma_tf32(dt, dbh + adv, dch + adv, idesc, 1u);
                        mma_tf32(dc, dbh + adv, dcl + adv, idesc, 1u);
                        mma_tf32(dc, dbl + adv, dch + adv, idesc, 1u);
                        mma_tf32(dc, dbl + adv, dcl + adv, idesc, 1u);
                    }
                    mma_commit(&bt_empty[sb]);
                    mma_commit(&c_empty[sc]);
                    if (b == n_blk - 1) mma_commit(done);
                }
                first = false;
                __syncwarp();
            }
            if (!ok) break;
        }
    } else {
        // ---- generators / per-slot epilogue ----
        const int gt = threadIdx.x - 64;              // 0 .. 255
        const int P = NS / 16;                        // pairs per thread per block
        const int row = gt % NS;
        const int t0 = (gt / NS) * P;
        const float *xr = xrows + (size_t)row * XS;
        const int n_slots_k = n_blk * kBlkPairs;
        uint32_t gphase = 0;
        long long g = 0;
        for (int r = 0;; r++) {
            bool ok = true;
            const int cell = slots[row].cell;             // fixed for the whole pass
            const bool active = cell >= 0;
            const float2 *kbase = a.K32 + (size_t)(active ? cell : 0) * n_slots_k + t0;
            if (P == 4) ok = gen_pass<4>(a, cring, cstride, kbase, xr, c_empty, c_full, &s_err, g, n_blk,
                                         SC, NS, row, t0, active, lane);
            else if (P == 2) ok = gen_pass<2>(a, cring, cstride, kbase, xr, c_empty, c_full, &s_err, g,
                                              n_blk, SC, NS, row, t0, active, lane);
            else ok = gen_pass<1>(a, cring, cstride, kbase, xr, c_empty, c_full, &s_err, g, n_blk, SC,
                                  NS, row, t0, active, lane);
            g += n_blk;
            if (!ok) break;
            // ---- epilogue: D (TMEM) -> smem [slot][bin] ----
            if (!wwait(done, r & 1, &s_err, ERR_WAIT_EPI)) break;
            tc_fence_after();
            float *Dsm = (float *)bring;                  // the mapping-tile ring is idle now
            const int DS = N;
            {
                const int q = warp & 3;                   // TMEM lane quadrant of this warp
                const int half = (warp - 2) >> 2;         // which half of the columns
                const int c0 = half * (NS / 2), c1 = c0 + NS / 2;
                const int bin = 32 * q + lane;
                for (int cc = c0; cc < c1; cc += 8) {
                    // compensated (Neumaier) FP32 sum of the accumulators
                    float sum[8], cmp[8];
#pragma unroll
                    for (int z = 0; z < 8; z++) { sum[z] = 0.f; cmp[z] = 0.f; }
                    for (int ch = 0; ch <= nacc; ch++) {
                        float v[8];
                        tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ch * NS + cc), v);
#pragma unroll
                        for (int z = 0; z < 8; z++) {
                            const float t = sum[z] + v[z];
                            cmp[z] += (fabsf(sum[z]) >= fabsf(v[z])) ? (sum[z] - t) + v[z] : (v[z] - t) + sum[z];
                            sum[z] = t;
                        }
                    }
                    if (bin < N) {
#pragma unroll
                        for (int z = 0; z < 8; z++)
                            if (cc + z < c1) Dsm[(size_t)(cc + z) * DS + bin] = sum[z] + cmp[z];
                    }
                }
            }
            tc_fence_before();
            if (!gen_sync(gbar, gphase, &s_err)) break;
            // ---- per-slot integrator logic ----
            for (int sidx = warp - 2; sidx < NS; sidx += kGenWarps) {
                Slot &sl = slots[sidx];
                if (sl.cell < 0) continue;
                Slot loc = sl;
                __syncwarp();
                bool fin = slot_advance(a, loc, xrows + (size_t)sidx * XS, Dsm + (size_t)sidx * DS, sidx);
                __syncwarp();
                if (fin) {
                    slot_finish(a, loc, sidx);
                    // refill from the global queue: cells 0 .. grid*NS-1 were the
                    // initial fill, later ones go to whichever slot frees first
                    int c = 0;
                    if (lane == 0) c = (int)gridDim.x * NS + atomicAdd(a.queue, 1);
                    c = __shfl_sync(0xffffffffu, c, 0);
                    __syncwarp();
                    if (lane == 0) sl = loc;
                    __syncwarp();
                    slot_load(a, sl, xrows + (size_t)sidx * XS, sidx, c < a.t.n_cells ? c : -1);
                } else if (lane == 0) {
                    sl = loc;
                }
                __syncwarp();
            }
            // generic-proxy writes to the stage memory (D staging) must be
            // ordered before the bulk copies of the next pass overwrite it
            fence_async_smem();
            if (!gen_sync(gbar, gphase, &s_err)) break;
            if (gt == 0) {
                int any = 0;
                for (int s2 = 0; s2 < NS; s2++) any |= (slots[s2].cell >= 0);
                s_continue = any;
                mbar_arrive(go);
            }
            if (!gen_sync(gbar, gphase, &s_err)) break;
            if (!s_continue) break;
        }
    }
    if (warp == 1 && lane == 0) {
        // every MMA this thread issued has completed before TMEM is freed
        mma_commit(fin);
        mbar_wait(fin, 0, &s_err, ERR_WAIT_MMA);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
    if (threadIdx.x == 0 && s_err) atomicCAS(a.err, 0, s_err);
}

struct Config { int grid, NS, S, XS, SB, NB8; size_t smem; };


Config mixed_config(int n_cells, int N)
{
    int dev = 0, n_sm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    Config c;
    // every SM gets a CTA once there are 16 cells per SM; slots per CTA are
    // a multiple of 16 (the MMA N), at most 64
    c.grid = std::max(1, std::min(n_sm, (n_cells + 15) / 16));
    const int per = (n_cells + c.grid - 1) / c.grid;
    int NS = ((per + 15) / 16) * 16;
    NS = std::min(NS, 64);
    if (NS > 32) NS = 64;
    c.NS = NS;
    c.S = kCStages;
    const int n16 = ((N + 15) / 16) * 16;
    c.XS = n16 + 4;                              // rows 16 B aligned, 4 words off the bank period
    c.NB8 = ((N + 7) / 8) * 8;
    const size_t bstride = 2 * (size_t)c.NB8 * 128;
    const size_t cring = (size_t)kCStages * 2 * NS * 128;
    const size_t tail = (size_t)NS * c.XS * 4 + (size_t)NS * sizeof(Slot) + 8 * (2 * kMaxSB + 2 * kCStages + 4);
    const size_t budget = 232448 - 1024 - 2048;  // opt-in shared memory, alignment, static
    int SB = (int)((budget - cring - tail) / bstride);
    SB = std::min(SB, kMaxSB);
    // the D staging area (NS x N doubles) aliases the mapping-tile ring
    while ((size_t)SB * bstride < (size_t)NS * N * 8 && SB < kMaxSB) SB++;
    c.SB = SB;
    // the MMA reads all 128 tile rows: rows past NB8 of the last tile fall in
    // the bytes after the ring, which must stay inside the allocation
    const size_t ring_end = (size_t)SB * bstride;
    const size_t layout_end = ring_end + cring + tail;
    c.smem = 1024 + std::max(layout_end, ring_end + (size_t)kTileBytes);
    return c;
}

cudaError_t launch_mixed(const cudisc_coag_ctx *c, int mode, double *rho, double *drho, double t_span,
                         double *dt_cell, const double *replay_h, const long long *replay_n,
                         long long replay_stride)
{
    Config cf = mixed_config(c->n_cells, c->N);
    const size_t need = (size_t)cf.grid * cf.NS * 5 * (size_t)c->N * sizeof(double);
    if (need > c->work_bytes) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(step_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cf.smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(c->d_counter + 1, 0, 2 * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    MixedArgs a;
    a.t = c->tables();
    a.K32 = c->d_K32;
    a.rho = rho;
    a.drho = drho;
    a.t_span = t_span;
    a.dt_cell = dt_cell;
    a.rtol = c->p.rtol;
    a.atol_rel = c->p.atol_rel;
    a.max_steps = c->p.max_substeps;
    a.replay_h = replay_h;
    a.replay_n = replay_n;
    a.replay_stride = replay_stride;
    a.out = c->d_out;
    a.err = c->d_counter + 1;
    a.queue = c->d_counter + 2;
    a.work = c->d_work;
    a.rec_dt = mode == MODE_STEP ? c->rec_dt : nullptr;
    a.rec_cap = c->rec_cap;
    a.rec_n = mode == MODE_RHS ? nullptr : c->rec_n;
    a.rec_status = mode == MODE_RHS ? nullptr : c->rec_status;
    a.NS = cf.NS;
    a.S = cf.S;
    a.XS = cf.XS;
    a.SB = cf.SB;
    a.NB8 = cf.NB8;
    a.mode = mode;
    step_mixed_kernel<<<cf.grid, kThreads, cf.smem, c->stream>>>(a);
    return cudaGetLastError();
}

} // namespace

// ---- fixed-scratch variant -------------------------------------------------
// Scratch for cudisc_coag_step_static_scratch: the per-slot FP64 integrator
// state that the regular entry point keeps in the context's workspace.  It is
// a file-scope device array of fixed size, so every GPU that loads this
// library holds these 16 MiB until the process exits.  Host code must not
// pass the symbol itself to a kernel (on the host it only names a stand-in);
// the device address comes from cudaGetSymbolAddress, taken once per device.
namespace {
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};
} // namespace

size_t static_scratch_bytes() { return kStaticScratchBytes; }

cudaError_t launch_step_mixed_static(const cudisc_coag_ctx *c, double *rho, double t_span,
                                     double *dt_cell, bool *too_big)
{
    *too_big = false;
    Config cf = mixed_config(c->n_cells, c->N);
    const size_t need = (size_t)cf.grid * cf.NS * 5 * (size_t)c->N * sizeof(double);
    if (need > kStaticScratchBytes) { *too_big = true; return cudaSuccess; }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    void *scratch = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess) return e;
            g_scratch_ptr[dev] = ptr;
        }
        scratch = g_scratch_ptr[dev];
    }
    e = cudaFuncSetAttribute(step_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cf.smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(c->d_counter + 1, 0, 2 * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    MixedArgs a;
    a.t = c->tables();
    a.K32 = c->d_K32;
    a.rho = rho;
    a.drho = nullptr;
    a.t_span = t_span;
    a.dt_cell = dt_cell;
    a.rtol = c->p.rtol;
    a.atol_rel = c->p.atol_rel;
    a.max_steps = c->p.max_substeps;
    a.replay_h = nullptr;
    a.replay_n = nullptr;
    a.replay_stride = 0;
    a.out = c->d_out;
    a.err = c->d_counter + 1;
    a.queue = c->d_counter + 2;
    a.work = (double *)scratch;     // every slot is written before it is read
    a.rec_dt = c->rec_dt;
    a.rec_cap = c->rec_cap;
    a.rec_n = c->rec_n;
    a.rec_status = c->rec_status;
    a.NS = cf.NS;
    a.S = cf.S;
    a.XS = cf.XS;
    a.SB = cf.SB;
    a.NB8 = cf.NB8;
    a.mode = MODE_STEP;
    step_mixed_kernel<<<cf.grid, kThreads, cf.smem, c->stream>>>(a);
    return cudaGetLastError();
}

size_t mixed_workspace_bytes(int n_cells, int N)
{
    Config cf = mixed_config(n_cells, N);
    return (size_t)cf.grid * cf.NS * 5 * (size_t)N * sizeof(double);
}

cudaError_t launch_rhs_mixed(const cudisc_coag_ctx *c, const double *rho, double *drho)
{
    return launch_mixed(c, MODE_RHS, const_cast<double *>(rho), drho, 1.0, nullptr, nullptr, nullptr, 0);
}

cudaError_t launch_step_mixed(const cudisc_coag_ctx *c, double *rho, double t_span, double *dt_cell,
                              const double *replay_h, const long long *replay_n, long long replay_stride)
{
    return launch_mixed(c, replay_h ? MODE_REPLAY : MODE_STEP, rho, nullptr, t_span, dt_cell, replay_h,
                        replay_n, replay_stride);
}

} // namespace cdc
