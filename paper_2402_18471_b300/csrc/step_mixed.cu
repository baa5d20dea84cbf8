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
//   MMA M = 128 rows = 64 cell slots x {A_hi, A_lo}: the generated operand
//   A (x_i x_j K p, split into a TF32 hi part and the remainder lo) is
//   written by the generator warps straight into tensor memory, rows 0..63
//   the hi parts and rows 64..127 the lo parts of the same 64 slots.
//   MMA N = the bins padded to 16 (Bt, streamed as swizzled TF32 hi and lo
//   tiles by the bulk-copy engine into shared memory, the B operand).
//   K = 32 TF32 elements (16 pairs) per block, 8 per instruction.  Per K
//   step two MMAs: [A_hi; A_lo] x Bt_hi into one of several FP32
//   accumulators (a contiguous share of the blocks each) and [A_hi; A_lo] x
//   Bt_lo into one more; the four split products hi.hi, lo.hi, hi.lo and
//   lo.lo are the four row-halves of the two accumulators.  Up to 128 bins
//   the two products are one MMA of N = 2 NBP: the Bt_lo tile follows the
//   Bt_hi tile in shared memory, so [Bt_hi; Bt_lo] is one B operand, and each
//   accumulator holds both products side by side (half as many
//   instructions, each twice as long, keep the tensor pipe's short queue
//   full through the issuer's barrier checks).  The Bt tiles and the slots'
//   K tables pass through shared memory (bulk copies in, MMA and generator
//   reads out).
// Warp roles: warp 0 bulk-copy producer, warp 1 MMA issuer and TMEM owner,
// warps 2..9 generate A (two warps per TMEM lane quadrant, one per half of a
// block's pairs) and, between right-hand sides, run the per-slot logic: the
// Bogacki-Shampine 3(2) stages, the error norm, step control, the state
// update with its mass budget, and refilling a slot with the next cell when
// one finishes.  (Sixteen generator warps measured 2 % slower once the K
// tables came from shared memory: the MMA-issuing thread shares its
// scheduler with the generators of its quadrant.)
//
// Every mbarrier wait is bounded by a clock limit; a wait that runs out
// records an error code in the status word and the kernel winds down.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <mutex>

#include "coag_internal.h"

namespace cdc {
namespace {

constexpr int kGenWarps = 8;                      // generator warps, kGenQ per TMEM lane quadrant
constexpr int kGenQ = kGenWarps / 4;
constexpr int kGP = kBlkPairs / kGenQ;            // pairs of each block a generator thread makes
constexpr int kGC = kGP / 2;                      // its 2-pair chunks of the K table
constexpr int kSlots = 64;                        // cell slots per CTA (TMEM rows / 2)
constexpr int kAStages = 3;                       // generated-operand stages in TMEM (two blocks, 64 columns each)
constexpr int kMaxMain = 8;                       // TMEM accumulators for the products with Bt_hi
constexpr int kMaxSB = 8;                         // mapping-tile ring depth (stages of two blocks), at most
constexpr int kMaxKS = 4;                         // K-table ring depth (stages of two blocks), at most
constexpr int kPrefetchK = 2;                     // K-table stages prefetched into L2 ahead of the ring,
                                                  // when the groups' K tables exceed L2
constexpr int kKBlkBytes = 16 * 8 * 64;           // K tables of one block for 64 slots: 8 chunks x 64 x 16 B
constexpr int kThreads = 64 + 32 * kGenWarps;
constexpr int kLaneBins = (kMaxMixedBins + 31) / 32;   // bins per lane in the per-slot logic
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz
constexpr long long kDrainCycles = 4000000000LL;  // ~2 s: drains of issued copies and MMAs
constexpr double A21 = 0.5, A32 = 0.75;
constexpr double B1 = 2.0 / 9.0, B2 = 1.0 / 3.0, B3 = 4.0 / 9.0;
constexpr double E1 = -5.0 / 72.0, E2 = 1.0 / 12.0, E3 = 1.0 / 9.0, E4 = -1.0 / 8.0;

enum Mode { MODE_STEP = 0, MODE_RHS = 1, MODE_REPLAY = 2 };
enum ErrCode { ERR_WAIT_PRODUCER = 1, ERR_WAIT_MMA = 2, ERR_WAIT_GEN = 3, ERR_WAIT_EPI = 4, ERR_WAIT_PEER = 5 };

struct MixedArgs {
    DevTables t;
    const float4 *K32;          // [n_cells][n_blk * 8] 2-pair chunks (k32_index)
    float4 *Kslot;              // [groups][n_blk][8][64]: the tables of the cells in each group's slots
    double *rho;                // state in/out (STEP, REPLAY) or input (RHS)
    double *drho;               // output (RHS)
    double t_span;
    double *dt_cell;
    double rtol, atol_rel;
    float rtol_f;
    long long max_steps;
    const double *replay_h;
    const long long *replay_n;
    long long replay_stride;
    CellOut *out;
    int *err;                   // device status word
    int *queue;                 // global work-queue head (cells past the initial fill)
    float *work;                // [groups][NS][5][N] slot state (see SlotBufs)
    double *rec_dt;
    long long rec_cap;
    long long *rec_n;
    int *rec_status;
    int NS, XS, mode;
    int SB, NBP;                // mapping-tile ring depth; bins padded to 16 (MMA N, tile rows copied)
    int kC;                     // initial cells per group (slot s of group x starts with cell x + s G)
    int KS;                     // K-table ring depth
    int sst_off;                // byte offset of the per-slot state in shared memory, or -1: in work
    WorkList wl;                // the cells to integrate (work item -> cell) and their spans
    int P;                      // CTAs per group of slots (a cluster of 1, 2, 4 or 8; see the kernel)
    int nacc;                   // TMEM accumulators for the products with Bt_hi (stacked: with [Bt_hi; Bt_lo])
    int stacked;                // 1: one MMA of N = 2 NBP takes Bt_hi and Bt_lo together (2 NBP <= 256)
    int pair;                   // 1: CTA pairs share M = 256 MMAs (two groups of slots per pair, see the kernel)
    long long wait_cycles;      // clock limit of the bounded waits (kWaitCycles; shorter only in tests)
    int withhold;               // test hook: 1 = the producer issues no copies, so the waits run out
    int prefetch_k;             // K-table stages prefetched into L2 ahead of the ring (0: none)
};

struct __align__(16) Slot {
    double t, h, hs, S, Sx, tend;      // tend: the cell's span
    long long nacc, nrej, nrep;
    float sxf, atolx, hsf;             // Sx, atol / Sx and hs in FP32 for the per-bin work
    int cell, phase, last, status;
    int kcell;                         // the cell whose K table this CTA last copied into its block
                                       // range of the group's buffer for this slot (-1: none)
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
// The clock limit of every bounded wait of this CTA (kWaitCycles unless a
// test shortened it through the arguments), set before the first wait.
__shared__ long long s_wait_lim;

// Bounded wait: false when the clock limit runs out or another role failed.
// Waiting threads back off a little between tests, leaving issue slots to
// the warps that work (the MMA issuer shares a scheduler with generators).
__device__ __noinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *s_err, int code)
{
    const long long t0 = clock64();
    for (int it = 0;; ++it) {
        if (mbar_test(b, parity)) return true;
        if (it >= 2) __nanosleep(32);
        if ((it & 63) == 63) {
            if (*s_err) return false;
            if (clock64() - t0 > s_wait_lim) { atomicCAS((int *)s_err, 0, code); return false; }
        }
    }
}
// Wait for asynchronous work this thread issued (bulk copies, MMAs) before
// the CTA frees what that work writes: unlike mbar_wait it does not give up
// when another role has failed, only after its own limit (kDrainCycles).
__device__ __noinline__ void mbar_drain(uint64_t *b, uint32_t parity)
{
    const long long t0 = clock64();
    for (int it = 0;; ++it) {
        if (mbar_test(b, parity)) return;
        __nanosleep(64);
        if ((it & 63) == 63 && clock64() - t0 > kDrainCycles) return;
    }
}
// ---- cluster (CTA pair) helpers ----
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// shared::cluster address of the same shared location in CTA `rank`
__device__ __forceinline__ uint32_t mapa(uint32_t saddr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_v4(uint32_t addr, float a, float b, float c, float d)
{
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}
__device__ __forceinline__ void st_cluster_s32(uint32_t addr, int v)
{
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_cluster() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }
// arrive on an mbarrier of another CTA of the cluster, releasing this thread's (and, after
// a __syncwarp, its warp's) prior writes at cluster scope
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_test_cluster(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(su32(b)), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded warp-wide wait for data other CTAs of the cluster released (acquire at cluster scope).
__device__ __noinline__ bool cwait(uint64_t *b, uint32_t parity, volatile int *s_err, int code)
{
    const long long t0 = clock64();
    for (int it = 0;; ++it) {
        if (__all_sync(0xffffffffu, mbar_test_cluster(b, parity))) return true;
        if (it >= 2) __nanosleep(32);
        if ((it & 63) == 63) {
            if (*s_err) return false;
            if (clock64() - t0 > s_wait_lim) { atomicCAS((int *)s_err, 0, code); return false; }
        }
    }
}
// Single-thread bounded wait for an mbarrier that other CTAs of the cluster
// arrive on (acquire at cluster scope).
__device__ __noinline__ bool twait_cluster(uint64_t *b, uint32_t parity, volatile int *s_err, int code)
{
    const long long t0 = clock64();
    for (int it = 0;; ++it) {
        if (mbar_test_cluster(b, parity)) return true;
        if (it >= 2) __nanosleep(32);
        if ((it & 63) == 63) {
            if (*s_err) return false;
            if (clock64() - t0 > s_wait_lim) { atomicCAS((int *)s_err, 0, code); return false; }
        }
    }
}
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Single-thread wait with the common already-complete case inline.
__device__ __forceinline__ bool twait(uint64_t *b, uint32_t parity, volatile int *s_err, int code)
{
    return mbar_test(b, parity) || mbar_wait(b, parity, s_err, code);
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
// Bulk prefetch of global memory into L2 (no destination, no completion)
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
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
// tcgen05.mma kind::tf32 with the A operand in tensor memory (M rows =
// lanes, K columns) and B in shared memory (descriptor).
__device__ __forceinline__ void mma_tf32_ts(uint32_t dt, uint32_t at, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
                 ::"r"(dt), "r"(at), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
// The same, accumulating into D (enable-input-d given as an immediate).
__device__ __forceinline__ void mma_tf32_ts_acc(uint32_t dt, uint32_t at, uint64_t b, uint32_t idesc)
{
    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;"
                 ::"r"(dt), "r"(at), "l"(b), "r"(idesc) : "memory");
}
// The same for a CTA pair (cta_group::2, issued by the even CTA): M = 256
// rows, rows 0..127 from this CTA's tensor memory and 128..255 from the odd
// CTA's at the same address; B's N rows split in two halves at the same
// shared-memory address of the two CTAs; D in each CTA's own tensor memory.
__device__ __forceinline__ void mma2_tf32_ts(uint32_t dt, uint32_t at, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::2.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
                 ::"r"(dt), "r"(at), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
// Store 8 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ __attribute__((unused)) void tmem_st8(uint32_t taddr, const float (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                   "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])),
                   "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}
// Store 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ __attribute__((unused)) void tmem_st16(uint32_t taddr, const float (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,"
                 "%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                   "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])),
                   "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
                   "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
                   "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
                   "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
                 : "memory");
}
// The generator's row store: 2 kGP columns (the other width is unused).
template <int W> __device__ __forceinline__ void tmem_st_row(uint32_t taddr, const float (&v)[W])
{
    if constexpr (W == 8) tmem_st8(taddr, v);
    else tmem_st16(taddr, v);
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(su32(bar)) : "memory");
}
// Completion of this pair's MMAs, signalled on the mbarrier at the same
// shared-memory offset in both CTAs of the pair (mask: their cluster ranks).
__device__ __forceinline__ void mma_commit2(uint64_t *bar, uint16_t mask)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
                 ::"r"(su32(bar)), "h"(mask) : "memory");
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
// TF32 split: hi = v rounded to nearest at 11 significant bits, an exact
// TF32 value, and lo = v - hi, exact in FP32 (|lo| <= 2^-11 |v|).  The tensor
// core reads lo at TF32 precision (its 13 low mantissa bits take no part), an
// error of at most 2^-10 |lo|, so the hi + lo it multiplies matches v to
// 2^-21 relative.  (Rounding lo as well would halve that bound for more
// arithmetic per element on the generators.)  The generators form hi by
// Veltkamp's split (gen_vals).

// ---- per-slot logic (one warp per slot, lanes over bins) ------------------

// Dynamic shared memory of the kernel (aligned to 1024 B where it is used).
extern __shared__ __align__(1024) uint8_t smem_raw[];
__device__ __forceinline__ uint8_t *smem_base()
{
    return (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
}

// The slot group this CTA serves.  Groups of P CTAs (a cluster of P); in
// pair mode a cluster of P pairs serves two groups, the even CTAs of the
// pairs group 2 x + 0 and the odd ones group 2 x + 1 (cluster ranks follow
// blockIdx.x in a one-dimensional cluster).
__device__ __forceinline__ int group_of_block(const MixedArgs &a)
{
    if (!a.pair) return (int)blockIdx.x / a.P;
    return ((int)blockIdx.x / (2 * a.P)) * 2 + ((int)blockIdx.x & 1);
}

// Slot state (5 N floats per slot kept by this CTA), in shared memory when
// it fits beside the rings, else in global scratch: the state y / Sx as an unevaluated float pair yh + yl (48 significant
// bits; yh, the state rounded to FP32, is also the stage input), and the stage
// right-hand sides in the same scaled units (kx = f / Sx = Sx D).  B300
// executes FP64 at a small fraction of its FP32 rate, so the per-step work
// stays in FP32: the stage inputs, error norm and step controller (their
// rounding sits below the contraction's own ~3e-7) and the state update,
// where error-free FP32 transformations keep the pair exact to 2^-48 and
// the mass budget of every accepted increment holds to that level.  FP64
// only carries the time, the step size and the cell's conversion at load and
// finish.
struct SlotBufs { float *yh, *yl, *k1, *k2, *k3; };

__device__ __forceinline__ SlotBufs slot_bufs(const MixedArgs &a, int slot)
{
    const int N = a.t.N;
    float *f;
    if (a.sst_off >= 0) {
        // the CTA keeps slots SL r .. SL r + SL - 1: index slot mod SL
        const int SL = a.NS / a.P;
        f = (float *)(smem_base() + a.sst_off) + (size_t)(slot % SL) * 5 * N;
    } else {
        f = a.work + ((size_t)group_of_block(a) * a.NS + slot) * 5 * (size_t)N;
    }
    return {f, f + N, f + 2 * N, f + 3 * N, f + 4 * N};
}

// s + e = a + b exactly (Knuth's TwoSum; explicit roundings so that no
// operation is fused or reassociated).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (h, l) += x for an unevaluated pair h + l with |l| <= ulp(h) / 2.
__device__ __forceinline__ void pair_add(float &h, float &l, float x)
{
    float s, e;
    two_sum(h, x, s, e);
    two_sum(s, __fadd_rn(e, l), h, l);
}

// Copy 2-pair chunks c_lo .. c_hi - 1 of cell c's K table into slot s's
// column of group grp's buffer ([block][chunk][slot] x 16 B, read by the
// producer's bulk copies, one per block).  The caller's threads t = 0 ..
// nthr - 1 take every nthr-th chunk, D loads in flight each.  Each CTA of a
// slot group copies the block range it streams, so that only its own
// producer reads what it wrote: the caller orders the stores before those
// copies with fence_proxy_global and a barrier.
static_assert(kSlots == 64, "the per-pass K-copy mask reads slots lane and lane + 32");
template <int D>
__device__ void copy_k_range(const MixedArgs &a, int grp, int s, int c, int c_lo, int c_hi, int t, int nthr)
{
    const int n_ch = a.t.n_blk * 8;
    const float4 *src = a.K32 + (size_t)c * n_ch;
    float4 *dst = a.Kslot + (size_t)grp * n_ch * kSlots + s;
    for (int i0 = c_lo + t; i0 < c_hi; i0 += D * nthr) {
        float4 v[D];
#pragma unroll
        for (int j = 0; j < D; j++) {
            const int i = i0 + j * nthr;
            v[j] = i < c_hi ? __ldg(src + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < D; j++) {
            const int i = i0 + j * nthr;
            if (i < c_hi) dst[(size_t)i * kSlots] = v[j];
        }
    }
}
__device__ __forceinline__ void fence_proxy_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Load cell c into slot: state, scales, phase 0 (or mark the slot empty).
// Its K table is copied afterwards (kcell = -1 until then): by the refilling
// warp in a lone CTA, else by every member, its own block range, after the
// stage-input exchange.
// owner = false: only the stage-input row and the cell id (a slot whose
// integrator state another CTA of the cluster keeps).
__device__ void slot_load(const MixedArgs &a, Slot &sl, float *xrow, int slot, int c, bool owner = true)
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
        s += v;
        sa += fabs(v);
    }
    s = warp_sum(s);
    sa = warp_sum(sa);
    const double Sx = sa > 0.0 ? sa : 1.0;
    const double r = 1.0 / Sx;
    for (int k = lane; k < a.XS; k += 32) {
        float h = 0.f;
        if (k < N) {
            const double z = rc[k] * r;
            h = (float)z;
            if (owner) {
                B.yh[k] = h;
                B.yl[k] = (float)(z - (double)h);
            }
        }
        xrow[k] = h;
    }
    if (lane == 0) {
        sl.cell = c;
        sl.phase = 0;
        sl.S = s;
        sl.Sx = Sx;
        sl.sxf = (float)Sx;
        sl.atolx = (float)(a.atol_rel * s * r);
        sl.t = 0.0;
        sl.tend = a.wl.spans ? a.wl.spans[c] : a.t_span;
        sl.h = (a.mode == MODE_STEP && a.dt_cell) ? a.dt_cell[c] : 0.0;
        sl.hs = 0.0;
        sl.hsf = 0.f;
        sl.nacc = sl.nrej = sl.nrep = 0;
        sl.last = 0;
        sl.status = CUDISC_OK;
        sl.kcell = -1;
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
        for (int k = lane; k < N; k += 32) {
            const double v = sl.Sx * ((double)B.yh[k] + (double)B.yl[k]);
            rc[k] = v;
            s1 += v;
        }
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

// Accept an increment dx (scaled units) into the state pair: the residual
// s = sum_k dx_k is moved in proportion to |dx_k| (mass budget), y += dx_k -
// q |dx_k| with q = s / sum_k |dx_k|, both terms added exactly.  s is summed
// as an exact float pair; sum_k |dx_k| in FP32 (relative error below N
// 2^-24), so the budget leaves at most that fraction of s, itself the
// contraction's rounding (~1e-7 of sum |dx|): ~1e-12 of the increment per
// step at worst.  yh, the new leading part, is the next stage input.
template <int MB>
__device__ void commit_increment(SlotBufs B, int N, const float *dx)
{
    const int lane = threadIdx.x & 31;
    float sh = 0.f, sl = 0.f, sa = 0.f;
#pragma unroll
    for (int m = 0; m < MB; m++) {                 // dx is 0 beyond N
        float e;
        two_sum(sh, dx[m], sh, e);
        sl = __fadd_rn(sl, e);
        sa = __fadd_rn(sa, fabsf(dx[m]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
        sa = __fadd_rn(sa, __shfl_xor_sync(0xffffffffu, sa, o));
        float e;
        two_sum(sh, oh, sh, e);
        sl = __fadd_rn(sl, __fadd_rn(ol, e));
    }
    const float q = sa > 0.f ? __fdiv_rn(__fadd_rn(sh, sl), sa) : 0.f;
#pragma unroll
    for (int m = 0; m < MB; m++) {
        const int k = lane + 32 * m;
        if (k < N) {
            float h = B.yh[k], l = B.yl[k];
            pair_add(h, l, dx[m]);
            pair_add(h, l, -__fmul_rn(q, fabsf(dx[m])));
            B.yh[k] = h;
            B.yl[k] = l;
        }
    }
    __syncwarp();
}

// First stage input x = yh + hs A21 k1 after choosing the step (shared by
// the first step and every step after an accept or reject).
__device__ bool begin_step(const MixedArgs &a, Slot &sl, float *xrow, SlotBufs B)
{
    const int N = a.t.N, lane = threadIdx.x & 31;
    if (sl.nacc + sl.nrej >= a.max_steps) { sl.status = CUDISC_EMAXSTEPS; return false; }
    sl.last = (sl.h >= sl.tend - sl.t);
    sl.hs = sl.last ? (sl.tend - sl.t) : sl.h;
    sl.hsf = (float)sl.hs;
    const float c1 = sl.hsf * (float)A21;
    for (int k = lane; k < N; k += 32) xrow[k] = B.yh[k] + c1 * B.k1[k];
    sl.phase = 1;
    return true;
}

// Process one right-hand side result, D = sum of the TMEM accumulators for
// this slot (kx = Sx D in scaled units).  Returns true when the slot
// finished its cell.
// MB: bins per lane, ceil(N / 32) (4 up to 128 bins, else kLaneBins).
template <int MB>
__device__ bool slot_advance(const MixedArgs &a, Slot &sl, float *xrow, const float *Drow, int slot)
{
    const int N = a.t.N, lane = threadIdx.x & 31;
    SlotBufs B = slot_bufs(a, slot);
    const float sx = sl.sxf;
    float kv[MB];
#pragma unroll
    for (int m = 0; m < MB; m++) {
        const int k = lane + 32 * m;
        kv[m] = (k < N) ? sx * Drow[k] : 0.f;
    }
    if (a.mode == MODE_RHS) {
        // d rho / dt = Sx^2 D with the FP64 mass budget (one pass, no state)
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
            for (int k = lane; k < N; k += 32) xrow[k] = B.yh[k] + c1 * B.k1[k];
            sl.phase = 1;
        } else if (sl.phase == 1) {
            const float c2 = (float)(hh * A32);
            for (int k = lane; k < N; k += 32) xrow[k] = B.yh[k] + c2 * B.k2[k];
            sl.phase = 2;
        } else {
            const float b1 = (float)(hh * B1), b2 = (float)(hh * B2), b3 = (float)(hh * B3);
            float dx[MB];
#pragma unroll
            for (int m = 0; m < MB; m++) {
                const int k = lane + 32 * m;
                dx[m] = (k < N) ? b1 * B.k1[k] + b2 * B.k2[k] + b3 * B.k3[k] : 0.f;
            }
            commit_increment<MB>(B, N, dx);
            sl.nrep++;
            sl.nacc = sl.nrep;
            if (sl.nrep >= nh) return true;
            for (int k = lane; k < N; k += 32) xrow[k] = B.yh[k];
            sl.phase = 0;
        }
        return false;
    }
    // adaptive Bogacki-Shampine 3(2)
    switch (sl.phase) {
    case 0: {
        if (!(sl.h > 0.0)) {
            const float atolx = sl.atolx;
            float q = INFINITY;
            for (int k = lane; k < N; k += 32)
                if (B.k1[k] != 0.f) q = fminf(q, (fabsf(B.yh[k]) + atolx) / fabsf(B.k1[k]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) q = fminf(q, __shfl_xor_sync(0xffffffffu, q, o));
            sl.h = isfinite(q) ? 0.1 * (double)q : sl.tend;
            if (sl.h > sl.tend) sl.h = sl.tend;
        }
        return !begin_step(a, sl, xrow, B);
    }
    case 1: {
        const float c2 = sl.hsf * (float)A32;
        for (int k = lane; k < N; k += 32) xrow[k] = B.yh[k] + c2 * B.k2[k];
        sl.phase = 2;
        return false;
    }
    case 2: {
        const float hf = sl.hsf;
        const float b1 = hf * (float)B1, b2 = hf * (float)B2, b3 = hf * (float)B3;
        for (int k = lane; k < N; k += 32)
            xrow[k] = B.yh[k] + (b1 * B.k1[k] + b2 * B.k2[k] + b3 * B.k3[k]);
        sl.phase = 3;
        return false;
    }
    default: {
        // phase 3: kv holds k4 = f(y1); y1 = yh + dx is the stage input
        const float hf = sl.hsf;
        const float b1 = hf * (float)B1, b2 = hf * (float)B2, b3 = hf * (float)B3;
        const float e1 = hf * (float)E1, e2 = hf * (float)E2, e3 = hf * (float)E3, e4 = hf * (float)E4;
        const float atolx = sl.atolx, rtol = a.rtol_f;
        float dx[MB];
        float E = 0.f;
        bool fin = true, pos = true;
#pragma unroll
        for (int m = 0; m < MB; m++) {
            const int k = lane + 32 * m;
            dx[m] = 0.f;
            if (k < N) {
                const float k1 = B.k1[k], k2 = B.k2[k], k3 = B.k3[k], yx = B.yh[k];
                dx[m] = b1 * k1 + b2 * k2 + b3 * k3;
                const float y1 = yx + dx[m];
                const float e = e1 * k1 + e2 * k2 + e3 * k3 + e4 * kv[m];
                const float sc = atolx + rtol * fmaxf(fabsf(yx), fabsf(y1));
                // the error ratio only decides accept/reject and the next
                // step, so the fast division serves; an empty cell (atol = 0,
                // y = 0) has no error, not 0/0
                const float r = e == 0.f ? 0.f : __fdividef(fabsf(e), sc);
                fin = fin && isfinite(r) && isfinite(y1);
                E = fmaxf(E, r);
                pos = pos && y1 >= -atolx;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) E = fmaxf(E, __shfl_xor_sync(0xffffffffu, E, o));
        const bool finite = __all_sync(0xffffffffu, fin);
        const bool nonneg = __all_sync(0xffffffffu, pos);
        if (finite && E <= 1.f && nonneg) {
            commit_increment<MB>(B, N, dx);
            sl.t = sl.last ? sl.tend : sl.t + sl.hs;
#pragma unroll
            for (int m = 0; m < MB; m++) {
                const int k = lane + 32 * m;
                if (k < N) B.k1[k] = kv[m];                 // FSAL
            }
            __syncwarp();
            if (lane == 0 && a.rec_dt && sl.nacc < a.rec_cap)
                a.rec_dt[(size_t)sl.cell * a.rec_cap + sl.nacc] = sl.hs;
            sl.nacc++;
            float fac = (E > 0.f) ? 0.9f * rcbrtf(E) : 5.f;
            fac = fminf(fmaxf(fac, 0.2f), 5.f);
            if (!(sl.last && sl.hs < sl.h)) sl.h = sl.hs * (double)fac;
            if (sl.t >= sl.tend) return true;
        } else {
            sl.nrej++;
            float fac;
            if (!finite) fac = 0.2f;
            else if (E > 1.f) fac = fmaxf(0.9f * rcbrtf(E), 0.2f);
            else fac = 0.5f;
            sl.h = sl.hs * (double)fac;
            if (sl.h < 1e-14 * sl.tend) { sl.status = finite ? CUDISC_EDTMIN : CUDISC_ENONFINITE; return true; }
        }
        return !begin_step(a, sl, xrow, B);
    }
    }
}

// Generator thread: one TMEM row (a slot's hi or lo part) and kGP pairs of
// every block (a kGenQ-th of its 16).  a = x_i x_j K p_coag, b = x_i x_j K
// p_frag, split into hi, v rounded to nearest at TF32's 11 significant bits,
// and lo = v - hi (exact); the thread keeps the half its row holds and
// writes the 2 kGP values into the stage's TMEM columns.  kv: the thread's
// 2-pair chunks {K p_c, K p_f, K p_c, K p_f}.
// Packed FP32 pairs (two lanes of one 64-bit register): one instruction
// rounds both products (mul/sub/fma.rn.f32x2, the same IEEE round-to-nearest
// as two scalar ones), halving the generators' FP32 issue.  The split is
// Veltkamp's (Dekker 1971): with t = (2^13 + 1) v, hi = t - (t - v) keeps the
// leading 24 - 13 = 11 bits of v, rounded to nearest.  It runs on the FMA
// pipe as three fused multiply-adds (t = sigma v - 0, d = v (-1) + t,
// hi = d (-1) + t): a chain of packed subtractions t - (t - v) came out as v
// itself (a probe found every lane's hi equal to v), and the one-instruction
// conversion cvt.rna.tf32.f32 runs on the conversion pipe, which bounded the
// generators (the three fused operations took the bench step from 58.3 to
// 55.8 ms).
__device__ __forceinline__ unsigned long long pk2(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

__device__ __forceinline__ void gen_vals(const float4 (&kc)[kGC], const float *xr, int bi, int jfirst,
                                         bool lo_half, float (&out)[2 * kGP])
{
    const float xi = xr[bi];
    float xj[kGP];
#pragma unroll
    for (int u = 0; u < kGP; u += 4) {
        const float4 x4 = *(const float4 *)(xr + jfirst + u);
        xj[u] = x4.x; xj[u + 1] = x4.y; xj[u + 2] = x4.z; xj[u + 3] = x4.w;
    }
    const float *kv = (const float *)kc;
    const unsigned long long xi2 = pk2(xi, xi);
    // Veltkamp's split constant 2^13 + 1, -1, and -0 (the addend that leaves t = sigma v)
    const unsigned long long sig2 = pk2(8193.0f, 8193.0f), mone2 = pk2(-1.0f, -1.0f), mzero2 = pk2(-0.0f, -0.0f);
#pragma unroll
    for (int u = 0; u < kGP; u += 2) {
        float xa, xb;
        upk2(mul2(xi2, pk2(xj[u], xj[u + 1])), xa, xb);          // x_i x_j of pairs u, u + 1
#pragma unroll
        for (int t = 0; t < 2; t++) {
            const float xx = t == 0 ? xa : xb;
            const int q = 2 * (u + t);
            const unsigned long long v2 = mul2(pk2(xx, xx), pk2(kv[q], kv[q + 1]));   // x_i x_j {K p_c, K p_f}
            const unsigned long long t2 = fma2(sig2, v2, mzero2);
            const unsigned long long h2 = fma2(mone2, fma2(mone2, v2, t2), t2);
            if (lo_half) upk2(sub2(v2, h2), out[q], out[q + 1]);
            else upk2(h2, out[q], out[q + 1]);
        }
    }
}

// One pass of a generator warp over its blocks, a stage of two a step.  The
// stage's K tables (all 64 slots, [block][chunk][slot] x 16 B) arrive in a
// shared-memory ring filled by the producer's bulk copies; a warp whose rows
// have no cell only takes part in the hand-overs (its TMEM rows feed
// accumulator rows nobody reads).
struct GenCtx {
    const MixedArgs *a;
    uint32_t tmem, lane_base;
    const uint8_t *kring;                // K ring: KS stages of 2 x kKBlkBytes
    const float *xr;
    uint64_t *c_empty, *c_full, *k_full, *k_empty;
    uint32_t c_full_remote;              // pair mode, odd CTA: the even CTA's c_full (0: arrive locally)
    volatile int *s_err;
    int n_blk, sub, lane, slot, KS;      // sub: which kGP pairs of each block
    bool lo_half, active;
    int bi, bj0;                         // pair row and first column of the next block
    int s, ks;                           // TMEM stage and K-ring stage of the next stage
    uint32_t u, ku;                      // their ring rounds
};

// One pipeline stage = two blocks (b = 2 st, 2 st + 1; the last stage of a
// pass may hold one): the wait for its K tables, their loads into registers
// and the release of the K ring stage, two products-and-splits, then the
// wait for its TMEM columns, the stores, one store wait and the arrival.
// The values are ready before the MMAs release the TMEM stage.
__device__ __forceinline__ bool gen_stage(GenCtx &G, int st, long long g)
{
    const int b = 2 * st;
    if (b >= G.n_blk) return true;
    const bool two = b + 1 < G.n_blk;
    int bi1 = G.bi, bj1 = G.bj0 + kBlkPairs;               // the second block's (i, j0)
    if (bj1 > bi1) { bi1++; bj1 = 0; }
    if (!wwait(&G.k_full[G.ks], G.ku & 1, G.s_err, ERR_WAIT_GEN)) return false;
    float oa[2 * kGP], ob[2 * kGP];
    // this thread's chunks 2 sub .. 2 sub + kGC - 1 of its slot, both blocks,
    // into registers; the ring stage is released before the products so that
    // the producer refills it a stage's arithmetic earlier
    float4 ka[kGC], kb[kGC];
    if (G.active) {
        const float4 *kp = reinterpret_cast<const float4 *>(G.kring + (size_t)G.ks * 2 * kKBlkBytes) +
                           (size_t)(kGC * G.sub) * kSlots + G.slot;
#pragma unroll
        for (int q = 0; q < kGC; q++) ka[q] = kp[q * kSlots];
#pragma unroll
        for (int q = 0; q < kGC; q++) kb[q] = two ? kp[kKBlkBytes / 16 + q * kSlots] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    if (G.lane == 0) mbar_arrive(&G.k_empty[G.ks]);
    if (G.active) {
        gen_vals(ka, G.xr, G.bi, G.bj0 + kGP * G.sub, G.lo_half, oa);
        if (two) gen_vals(kb, G.xr, bi1, bj1 + kGP * G.sub, G.lo_half, ob);
    }
    if (g >= kAStages && !wwait(&G.c_empty[G.s], (G.u + 1) & 1, G.s_err, ERR_WAIT_GEN)) return false;
    if (G.active) {
        tc_fence_after();
        const uint32_t base = G.tmem + G.lane_base + (uint32_t)(G.s * 64 + 2 * kGP * G.sub);
        tmem_st_row(base, oa);
        if (two) tmem_st_row(base + 32, ob);
        tmem_st_wait();
        tc_fence_before();
    }
    __syncwarp();
    if (G.lane == 0) {
        if (G.c_full_remote) mbar_arrive_remote(G.c_full_remote + 8u * (uint32_t)G.s);   // release, cluster scope
        else mbar_arrive(&G.c_full[G.s]);
    }
    // blocks run along rows: (i, 0), (i, 16), .. while j0 <= i, then (i + 1, 0)
    G.bi = bi1;
    G.bj0 = bj1 + kBlkPairs;
    if (G.bj0 > G.bi) { G.bi++; G.bj0 = 0; }
    if (++G.s == kAStages) { G.s = 0; G.u++; }
    if (++G.ks == G.KS) { G.ks = 0; G.ku++; }
    return true;
}

// Stages st_lo .. st_hi - 1 of a pass (blocks 2 st_lo .. min(n_blk, 2 st_hi) - 1);
// G.n_blk is the end of that block range.
__device__ __forceinline__ bool gen_pass(GenCtx &G, long long g0, int st_lo, int st_hi)
{
    const int b0 = 2 * st_lo;
    G.bi = __ldg(G.a->t.blk_i + b0);
    G.bj0 = __ldg(G.a->t.blk_j0 + b0);
    for (int st = st_lo; st < st_hi; st++)
        if (!gen_stage(G, st, g0 + (st - st_lo))) return false;
    return true;
}

// ---- the kernel --------------------------------------------------------------
//
// Each group of 64 slots is served by a cluster of P CTAs (P = 1, 2, 4 or
// 8).  All of them hold the stage inputs of all 64 slots and each streams a
// contiguous P-th of the stages of a pass (its tensor-core work divides by
// P); CTA r keeps the integrator state of slots SL r .. SL r + SL - 1 (SL =
// 64 / P).  After its MMAs a CTA sends the partial sums of the other CTAs'
// slots into their shared memory; after the per-slot logic it sends its own
// slots' new stage inputs and cells to all of them, and each member then
// copies its block range of the new cells' K tables.  Each exchange ends in
// one remote mbarrier arrival per sending warp and receiving CTA
// (release/acquire at cluster scope).  Smaller P loses less to the
// exchanges; larger P shortens a pass, which bounds the time of the costliest
// cells once there are fewer cells than slots to keep busy.

template <bool Pair, int MB>
__global__ void __launch_bounds__(kThreads, 1) step_mixed_kernel(MixedArgs a)
{
    uint8_t *sm = smem_base();
    const int NS = a.NS, XS = a.XS, N = a.t.N, n_blk = a.t.n_blk, NBP = a.NBP;
    const int SB = a.SB;
    const int P = a.P;                                  // CTAs per group (its members)
    constexpr bool pairm = Pair;                        // CTA pairs share M = 256 MMAs
    const int Q = pairm ? 2 * P : P;                    // cluster size
    const bool clustered = Q > 1;                       // cluster-wide barriers needed
    const bool xchg = P > 1;                            // partial sums and stage inputs exchanged
    const int crank = clustered ? (int)cluster_rank() : 0;
    const int half = pairm ? (crank & 1) : 0;           // pair mode: 0 = even CTA (issues the MMAs), 1 = odd
    const int rank = pairm ? (crank >> 1) : crank;      // this CTA's member index in its group
    const bool leader = half == 0;
    // cluster rank of member o of this CTA's group
    auto member = [&](int o) { return (uint32_t)(pairm ? 2 * o + half : o); };
    const uint16_t pair_mask = (uint16_t)(3u << (crank & ~1));
    const int ngrp = pairm ? ((int)gridDim.x / Q) * 2 : (int)gridDim.x / P;
    const int grp = group_of_block(a);
    const int SL = NS / P;                              // slots whose state this CTA keeps
    const int own0 = rank * SL;
    const int half_bytes = NBP * 128;                   // rows of one Bt tile copied
    // one block of tiles: hi then lo (pair mode: this CTA's half, hi rows in
    // the even CTA and lo rows in the odd one), 1024-aligned
    const int bstride = (((pairm ? 1 : 2) * half_bytes + 1023) / 1024) * 1024;
    const int sstride = 2 * bstride;                    // one stage: two blocks
    const int n_st = (n_blk + 1) / 2;                   // stages per pass
    const int st_lo = (int)((long long)rank * n_st / P);
    const int st_hi = (int)((long long)(rank + 1) * n_st / P);
    const int my_st = st_hi - st_lo;                    // >= 2 (the launch needs n_st >= 2 P)
    const int b_lo = 2 * st_lo, b_hi = min(n_blk, 2 * st_hi);
    const int KS = a.KS;
    uint8_t *bring = sm;                                // mapping tiles (also the D staging area)
    uint8_t *kring = bring + (size_t)SB * sstride;      // K tables of the slots, KS stages of two blocks
    // (per-slot state at sm + a.sst_off, after the K ring, when it is in shared memory)
    float *xrows = (float *)(kring + (size_t)KS * 2 * kKBlkBytes +
                             (a.sst_off >= 0 ? (size_t)SL * 5 * N * sizeof(float) : 0));
    float *dpeer = xrows + (size_t)NS * XS;             // [P-1][SL][NBP] partial sums from the others
    Slot *slots = (Slot *)(dpeer + (size_t)(P - 1) * SL * NBP);
    uint64_t *bars = (uint64_t *)(slots + NS);
    uint64_t *bt_full = bars, *bt_empty = bars + SB;
    uint64_t *c_full = bars + 2 * SB, *c_empty = bars + 2 * SB + kAStages;
    uint64_t *done = bars + 2 * SB + 2 * kAStages, *go = done + 1, *gbar = done + 2, *fin = done + 3;
    uint64_t *dx_full = done + 4, *xg_full = done + 5;
    uint64_t *k_full = done + 6, *k_empty = done + 6 + KS;
    uint64_t *pair_full = k_empty + KS;                 // [kGenWarps / 2]: a lo-row warp's sums are in Dlo
    // [SB] pair mode, even CTA: the odd one's tiles landed (indexed like the
    // tile ring: the odd CTA can relay stage g + SB only after this CTA's
    // commit for stage g released that ring slot, so one round at a time)
    uint64_t *pr_full = pair_full + kGenWarps / 2;
    uint64_t *cx_full = pr_full + kMaxSB;               // pair mode: the partner's continue flag arrived
    __shared__ uint32_t s_tmem;
    __shared__ int s_err, s_continue, s_any_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // TMEM columns: kAStages x 64 for the generated operand, then nacc
    // accumulators for [A_hi; A_lo] x Bt_hi (each a contiguous share of this
    // CTA's blocks, summed in the epilogue with a compensated FP32 sum) and
    // one for [A_hi; A_lo] x Bt_lo, NBP columns each; stacked, nacc
    // accumulators of 2 NBP columns for [A_hi; A_lo] x [Bt_hi; Bt_lo].  Either
    // way the epilogue sums nreg regions of NBP columns.
    const bool stacked = a.stacked != 0;
    const int nacc = a.nacc < b_hi - b_lo ? a.nacc : b_hi - b_lo;   // every accumulator gets a block
    const int nreg = stacked ? 2 * nacc : nacc + 1;
    const uint32_t acol = kAStages * 64;
    const int tcols = (int)acol + nreg * NBP;
    const uint32_t ncols = tcols <= 32 ? 32 : tcols <= 64 ? 64 : tcols <= 128 ? 128 : tcols <= 256 ? 256 : 512;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SB; s++) {
            mbar_init(&bt_full[s], 1);
            mbar_init(&bt_empty[s], 1);
        }
        for (int s = 0; s < kAStages; s++) {
            // pair mode: the even CTA's stage takes both CTAs' generators
            mbar_init(&c_full[s], pairm ? 2 * kGenWarps : kGenWarps);
            mbar_init(&c_empty[s], 1);
        }
        mbar_init(done, 1);
        mbar_init(go, 1);
        mbar_init(gbar, 32 * kGenWarps);
        mbar_init(fin, 1);
        // partial sums: the kGenQ hi-row warps of each other CTA whose rows
        // hold slots kept here; stage inputs: every generator warp of each
        // other CTA
        mbar_init(dx_full, xchg ? kGenQ * (P - 1) : 1);
        mbar_init(xg_full, xchg ? kGenWarps * (P - 1) : 1);
        for (int s = 0; s < KS; s++) {
            mbar_init(&k_full[s], 1);
            mbar_init(&k_empty[s], kGenWarps);
        }
        for (int s = 0; s < kGenWarps / 2; s++) mbar_init(&pair_full[s], 1);
        for (int s = 0; s < SB; s++) mbar_init(&pr_full[s], 1);
        mbar_init(cx_full, 1);
        s_err = 0;
        s_continue = 1;
        s_wait_lim = a.wait_cycles;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        if constexpr (Pair) {
            // both CTAs of the pair allocate together (the same columns in each)
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                         ::"r"(su32(&s_tmem)), "r"(ncols) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         ::"r"(su32(&s_tmem)), "r"(ncols) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    // initial slot fill: group x takes cells x, x + G, .., x + (C - 1) G (C =
    // the cells per group, at most NS): every group a spread of radii.  Every
    // CTA of the cluster sets up the stage inputs of all 64 slots and copies
    // its block range of their K tables into the group's buffer; the state
    // of each slot is set up by the one that keeps it.
    const int C = a.kC;
    const int n_work = a.wl.count ? *a.wl.count : a.t.n_cells;   // work item w is cell wl.cells[w] (or w)
    if (warp >= 2) {
        for (int s = warp - 2; s < NS; s += kGenWarps) {
            const int w = grp + s * ngrp;
            const int c = (s < C && w < n_work) ? (a.wl.cells ? a.wl.cells[w] : w) : -1;
            slot_load(a, slots[s], xrows + (size_t)s * XS, s, c, s >= own0 && s < own0 + SL);
            if (c >= 0) copy_k_range<16>(a, grp, s, c, 8 * b_lo, 8 * b_hi, lane, 32);
            __syncwarp();
            if (lane == 0) slots[s].kcell = c;
        }
        fence_proxy_global();
    }
    tc_fence_before();
    __syncthreads();
    if (clustered) cluster_sync_all();                // the others' barriers exist before any remote arrival
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        // ---- producer, one thread: the bulk-copy engine fills two rings, the
        // slots' K tables (needed first, by the generators; up to KS stages
        // ahead) and the mapping tiles (rows 0..NBP-1 of hi and lo, for the
        // MMAs; up to SB stages ahead).  Each ring is refilled as soon as its
        // oldest stage is released, without waiting on the other ----
        if (lane == 0) {
            long long g = 0, gk = 0;
            int ps = 0, ks = 0;
            uint32_t pu = 0, ku = 0;
            const float4 *kgrp = a.Kslot + (size_t)grp * n_blk * 8 * kSlots;   // this group's tables
            bool ok = a.withhold == 0;
            for (int r = 0; ok; r++) {
                if (r > 0) {
                    if (!twait(go, (r - 1) & 1, &s_err, ERR_WAIT_PRODUCER)) break;
                    if (!s_continue) break;
                }
                int nt = 0, nk = 0;                     // tile and K stages of this pass issued
                long long t_last = clock64();
                for (int it = 0; nt < my_st; it++) {
                    bool progress = false;
                    if (nk < my_st && (gk < KS || mbar_test(&k_empty[ks], (ku + 1) & 1))) {
                        const int sk = st_lo + nk;
                        const int nb = 2 * sk + 1 < n_blk ? 2 : 1;
                        mbar_expect_tx(&k_full[ks], (uint32_t)(nb * kKBlkBytes));
                        for (int q = 0; q < nb; q++)
                            bulk_g2s(kring + ((size_t)ks * 2 + q) * kKBlkBytes,
                                     kgrp + (size_t)(2 * sk + q) * 8 * kSlots, kKBlkBytes, &k_full[ks]);
                        if (a.prefetch_k > 0) {
                            // the K tables prefetch_k stages on (this CTA's range,
                            // wrapping into the next pass) into L2, so that their
                            // copy into the ring reads L2 rather than DRAM
                            int sp = sk + a.prefetch_k;
                            if (sp >= st_hi) sp = st_lo + (sp - st_hi);
                            if (sp < st_hi) {
                                const int nbp = 2 * sp + 1 < n_blk ? 2 : 1;
                                bulk_prefetch_l2(kgrp + (size_t)(2 * sp) * 8 * kSlots, (uint32_t)(nbp * kKBlkBytes));
                            }
                        }
                        nk++;
                        gk++;
                        if (++ks == KS) { ks = 0; ku++; }
                        progress = true;
                    }
                    if (nt < nk && (g < SB || mbar_test(&bt_empty[ps], (pu + 1) & 1))) {
                        const int st = st_lo + nt;
                        const int nb = 2 * st + 1 < n_blk ? 2 : 1;
                        mbar_expect_tx(&bt_full[ps], (uint32_t)(nb * (pairm ? 1 : 2) * half_bytes));
                        for (int q = 0; q < nb; q++) {
                            uint8_t *dst = bring + (size_t)ps * sstride + (size_t)q * bstride;
                            const uint8_t *src =
                                (const uint8_t *)(a.t.Btiles + (size_t)(2 * st + q) * (2 * half_bytes / 16));
                            if (pairm) {
                                // this CTA's rows of the stacked B operand: hi (even CTA) or lo (odd)
                                bulk_g2s(dst, src + (size_t)half * half_bytes, half_bytes, &bt_full[ps]);
                            } else {
                                bulk_g2s(dst, src, half_bytes, &bt_full[ps]);
                                bulk_g2s(dst + half_bytes, src + half_bytes, half_bytes, &bt_full[ps]);
                            }
                        }
                        nt++;
                        g++;
                        if (++ps == SB) { ps = 0; pu++; }
                        progress = true;
                    }
                    if (progress) {
                        t_last = clock64();
                    } else {
                        __nanosleep(32);
                        if ((it & 63) == 63) {
                            if (*(volatile int *)&s_err) { ok = false; break; }
                            if (clock64() - t_last > s_wait_lim) {
                                atomicCAS(&s_err, 0, ERR_WAIT_PRODUCER);
                                ok = false;
                                break;
                            }
                        }
                    }
                }
            }
            // every copy issued has landed before the CTA can leave: wait for
            // the last issued round of each ring stage (the rings only advance
            // on this thread's issues, so its parity is unambiguous)
            for (int q = 0; q < SB; q++)
                if (g > q) mbar_drain(&bt_full[q], (uint32_t)(((g - 1 - q) / SB) & 1));
            for (int q = 0; q < KS; q++)
                if (gk > q) mbar_drain(&k_full[q], (uint32_t)(((gk - 1 - q) / KS) & 1));
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer: one thread (the tensor pipe's queue is shallow, so
        // the issuing thread does nothing between MMAs that it can avoid).
        // Pair mode: the even CTA issues M = 256 MMAs for both CTAs; the odd
        // CTA's thread instead tells it, stage by stage, that its half of the
        // mapping tiles has landed (its generators arrive on the even CTA's
        // c_full themselves) ----
        if (lane == 0 && pairm && !leader) {
            const uint32_t pr_remote = mapa(su32(pr_full), (uint32_t)(crank ^ 1));
            int ms = 0;
            uint32_t mu = 0;
            for (int r = 0;; r++) {
                if (r > 0) {
                    if (!twait(go, (r - 1) & 1, &s_err, ERR_WAIT_MMA)) break;
                    if (!s_continue) break;
                }
                bool ok = true;
                for (int st = st_lo; st < st_hi; st++) {
                    const int sb = ms;
                    const uint32_t ub = mu;
                    if (++ms == SB) { ms = 0; mu++; }
                    if (!twait(&bt_full[sb], ub & 1, &s_err, ERR_WAIT_MMA)) { ok = false; break; }
                    mbar_arrive_remote(pr_remote + 8u * (uint32_t)sb);   // release, cluster scope
                }
                if (!ok) break;
            }
        } else if (lane == 0) {
            const uint32_t idesc = idesc_tf32(pairm ? 4 * kSlots : 2 * kSlots, stacked ? 2 * NBP : NBP);
            const int nb_mine = b_hi - b_lo;
            long long g = 0;
            int ms = 0, mc = 0;
            uint32_t mu = 0, mv = 0;
            for (int r = 0;; r++) {
                if (r > 0) {
                    if (!twait(go, (r - 1) & 1, &s_err, ERR_WAIT_MMA)) break;
                    if (!s_continue) break;
                }
                bool ok = true;
                int ch = 0, ch_next = (nb_mine + nacc - 1) / nacc;   // Bt_hi accumulator of the block
                bool first = true;
                const uint32_t dl = tmem + acol + (uint32_t)(nacc * NBP);
                for (int st = st_lo; st < st_hi; st++, g++) {
                    const int sb = ms, sc = mc;
                    const uint32_t ub = mu, uc = mv;
                    if (++ms == SB) { ms = 0; mu++; }
                    if (++mc == kAStages) { mc = 0; mv++; }
                    if (!twait(&bt_full[sb], ub & 1, &s_err, ERR_WAIT_MMA) ||
                        !(pairm ? twait_cluster(&c_full[sc], uc & 1, &s_err, ERR_WAIT_MMA)
                                : twait(&c_full[sc], uc & 1, &s_err, ERR_WAIT_MMA)) ||
                        (pairm && !twait_cluster(&pr_full[sb], ub & 1, &s_err, ERR_WAIT_PEER))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int nb = 2 * st + 1 < n_blk ? 2 : 1;
                    for (int q = 0; q < nb; q++) {
                        const int bl = 2 * st + q - b_lo;     // block index within this CTA's range
                        if (bl == ch_next) { ch++; ch_next = (int)(((long long)(ch + 1) * nb_mine + nacc - 1) / nacc); first = true; }
                        const uint32_t bt_hi = su32(bring + (size_t)sb * sstride + (size_t)q * bstride);
                        const uint64_t dbh = sw128_desc(bt_hi), dbl = sw128_desc(bt_hi + half_bytes);
                        const uint32_t at = tmem + (uint32_t)(sc * 64 + q * 32);
                        const uint32_t dh = tmem + acol + (uint32_t)(ch * (stacked ? 2 * NBP : NBP));
                        // the four K steps into one accumulator (stacked: both
                        // products at once), else then into the Bt_lo one
                        if constexpr (Pair) {
#pragma unroll
                            for (int kk = 0; kk < 4; kk++)
                                mma2_tf32_ts(dh, at + 8 * kk, dbh + 2 * kk, idesc, (first && kk == 0) ? 0u : 1u);
                            first = false;
                        } else {
                            mma_tf32_ts(dh, at, dbh, idesc, first ? 0u : 1u);
#pragma unroll
                            for (int kk = 1; kk < 4; kk++) mma_tf32_ts_acc(dh, at + 8 * kk, dbh + 2 * kk, idesc);
                            if (!stacked) {
                                mma_tf32_ts(dl, at, dbl, idesc, bl == 0 ? 0u : 1u);
#pragma unroll
                                for (int kk = 1; kk < 4; kk++) mma_tf32_ts_acc(dl, at + 8 * kk, dbl + 2 * kk, idesc);
                            }
                            first = false;
                        }
                    }
                    if constexpr (Pair) {
                        mma_commit2(&bt_empty[sb], pair_mask);
                        mma_commit2(&c_empty[sc], pair_mask);
                        if (st == st_hi - 1) mma_commit2(done, pair_mask);
                    } else {
                        mma_commit(&bt_empty[sb]);
                        mma_commit(&c_empty[sc]);
                        if (st == st_hi - 1) mma_commit(done);
                    }
                }
                if (!ok) break;
            }
        }
        __syncwarp();
    } else {
        // ---- generators / per-slot epilogue ----
        const int gt = threadIdx.x - 64;              // 0 .. 32 kGenWarps - 1
        const int qd = warp & 3;                      // TMEM lane quadrant of this warp
        const int row = 32 * qd + lane;               // TMEM row: slot (row & 63), hi or lo part
        const int slot = row & (kSlots - 1);
        const bool lo_half = row >= kSlots;
        const int sub = (warp - 2) / 4;               // pairs kGP sub .. kGP sub + kGP - 1 of each block
        const uint32_t lane_base = (uint32_t)(32 * qd) << 16;
        const float *xr = xrows + (size_t)slot * XS;
        // the CTA that keeps this row's slot, and where its partial sums go:
        // here [slot][bin], or that CTA's buffer [src][slot][bin] for source
        // index src (this CTA's rank among the others)
        const int owner = slot / SL;
        const bool rows_own = owner == rank;
        const int sl_row = slot - owner * SL;
        float *Dsm = (float *)bring;                  // [SL][NBP]; the mapping-tile ring is idle then
        float *Dlo = Dsm + (size_t)SL * NBP;          // [64][NBP]: the lo-row sums of every slot
        const int pair = (qd & 1) * kGenQ + sub;      // the hi-row / lo-row warp pair of these slots and columns
        const uint32_t d_remote = rows_own ? 0u :
            mapa(su32(dpeer), member(owner)) +
            (uint32_t)((size_t)((rank < owner ? rank : rank - 1) * SL) * NBP * 4);
        // owners of this warp's 32 consecutive slots
        const int own_lo = (slot - lane) / SL, own_hi = (slot - lane + 31) / SL;
        uint32_t gphase = 0;
        long long g = 0;
        GenCtx G;                                     // ring positions carry over between passes
        G.a = &a; G.tmem = tmem; G.lane_base = lane_base; G.kring = kring; G.xr = xr;
        G.c_empty = c_empty; G.c_full = c_full; G.k_full = k_full; G.k_empty = k_empty;
        G.c_full_remote = (pairm && !leader) ? mapa(su32(c_full), (uint32_t)(crank ^ 1)) : 0u;
        G.s_err = &s_err; G.n_blk = b_hi; G.sub = sub; G.lane = lane; G.slot = slot; G.KS = KS;
        G.lo_half = lo_half; G.active = false; G.bi = G.bj0 = 0;
        G.s = 0; G.ks = 0; G.u = 0; G.ku = 0;
        for (int r = 0;; r++) {
            const int cell = slots[slot].cell;        // fixed for the whole pass
            const bool active = __any_sync(0xffffffffu, cell >= 0);
            G.active = active;
            const bool ok = gen_pass(G, g, st_lo, st_hi);
            g += my_st;
            if (!ok) break;
            // ---- epilogue: D (TMEM) -> [slot][bin], here or in the owner.  The
            // lo-row warp of each column group leaves its sums in Dlo; the
            // hi-row warp of the same slots and columns adds them and sends
            // one row per slot ----
            if (!wwait(done, r & 1, &s_err, ERR_WAIT_EPI)) break;
            tc_fence_after();
            bool epi_ok = true;
            {
                bool got_lo = false;
                for (int cc = 8 * sub; cc < NBP; cc += 8 * kGenQ) {
                    // compensated (Neumaier) FP32 sum of the accumulators
                    float sum[8], cmp[8];
#pragma unroll
                    for (int z = 0; z < 8; z++) { sum[z] = 0.f; cmp[z] = 0.f; }
                    for (int ch = 0; ch < nreg; ch++) {
                        float v[8];
                        tmem_ld8(tmem + lane_base + acol + (uint32_t)(ch * NBP + cc), v);
#pragma unroll
                        for (int z = 0; z < 8; z++) {
                            const float t = sum[z] + v[z];
                            cmp[z] += (fabsf(sum[z]) >= fabsf(v[z])) ? (sum[z] - t) + v[z] : (v[z] - t) + sum[z];
                            sum[z] = t;
                        }
                    }
                    float o[8];
#pragma unroll
                    for (int z = 0; z < 8; z++) o[z] = sum[z] + cmp[z];
                    float *lo_at = Dlo + (size_t)slot * NBP + cc;
                    if (lo_half) {
                        *(float4 *)lo_at = make_float4(o[0], o[1], o[2], o[3]);
                        *(float4 *)(lo_at + 4) = make_float4(o[4], o[5], o[6], o[7]);
                        continue;
                    }
                    if (!got_lo) {
                        if (!wwait(&pair_full[pair], r & 1, &s_err, ERR_WAIT_EPI)) { epi_ok = false; break; }
                        got_lo = true;
                    }
                    const float4 la = *(const float4 *)lo_at, lb = *(const float4 *)(lo_at + 4);
                    o[0] += la.x; o[1] += la.y; o[2] += la.z; o[3] += la.w;
                    o[4] += lb.x; o[5] += lb.y; o[6] += lb.z; o[7] += lb.w;
                    const size_t off = (size_t)sl_row * NBP + cc;   // floats
                    if (rows_own) {
                        *(float4 *)(Dsm + off) = make_float4(o[0], o[1], o[2], o[3]);
                        *(float4 *)(Dsm + off + 4) = make_float4(o[4], o[5], o[6], o[7]);
                    } else {
                        st_cluster_v4(d_remote + (uint32_t)(off * 4), o[0], o[1], o[2], o[3]);
                        st_cluster_v4(d_remote + (uint32_t)(off * 4 + 16), o[4], o[5], o[6], o[7]);
                    }
                }
                if (lo_half) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&pair_full[pair]);
                } else if (epi_ok) {
                    if (!got_lo && !wwait(&pair_full[pair], r & 1, &s_err, ERR_WAIT_EPI)) epi_ok = false;
                    if (epi_ok && xchg) {
                        // one arrival at every other CTA whose slots this warp's rows hold
                        fence_cluster();
                        __syncwarp();
                        if (lane == 0)
                            for (int o = own_lo; o <= own_hi; o++)
                                if (o != rank) mbar_arrive_remote(mapa(su32(dx_full), member(o)));
                    }
                }
            }
            if (!epi_ok) break;
            tc_fence_before();
            if (xchg && !cwait(dx_full, r & 1, &s_err, ERR_WAIT_PEER)) break;
            if (!gen_sync(gbar, gphase, &s_err)) break;
            // ---- per-slot integrator logic for the slots kept here ----
            for (int sl = warp - 2; sl < SL; sl += kGenWarps) {
                const int sidx = own0 + sl;
                Slot &slr = slots[sidx];
                // D = sum of the partial rows (here, then from the others)
                float *Drow = Dsm + (size_t)sl * NBP;
                if (xchg) {
                    // the members' partial rows added in member order (not
                    // starting with this CTA's own), so that a cell's result
                    // does not depend on which member keeps its slot
                    float v[MB];
#pragma unroll
                    for (int m = 0; m < MB; m++) v[m] = 0.f;
                    for (int o = 0; o < P; o++) {
                        const float *dp = o == rank ? Drow : dpeer + ((size_t)(o < rank ? o : o - 1) * SL + sl) * NBP;
#pragma unroll
                        for (int m = 0; m < MB; m++)
                            if (lane + 32 * m < N) v[m] = o == 0 ? dp[lane + 32 * m] : v[m] + dp[lane + 32 * m];
                    }
#pragma unroll
                    for (int m = 0; m < MB; m++)
                        if (lane + 32 * m < N) Drow[lane + 32 * m] = v[m];
                }
                __syncwarp();
                if (slr.cell >= 0) {
                    Slot loc = slr;
                    __syncwarp();
                    bool fin = slot_advance<MB>(a, loc, xrows + (size_t)sidx * XS, Drow, sidx);
                    __syncwarp();
                    if (fin) {
                        slot_finish(a, loc, sidx);
                        // refill from the global queue: cells 0 .. G*C-1 were the
                        // initial fill, later ones go to whichever slot frees first
                        int w = 0;
                        if (lane == 0) w = ngrp * C + atomicAdd(a.queue, 1);
                        w = __shfl_sync(0xffffffffu, w, 0);
                        // the queue's next two cells (loaded here, used after
                        // this refill, so that their latency overlaps it)
                        int cn[2];
#pragma unroll
                        for (int d = 0; d < 2; d++)
                            cn[d] = w + 1 + d < n_work ? (a.wl.cells ? a.wl.cells[w + 1 + d] : w + 1 + d) : -1;
                        __syncwarp();
                        if (lane == 0) slr = loc;
                        __syncwarp();
                        const int cnew = w < n_work ? (a.wl.cells ? a.wl.cells[w] : w) : -1;
                        slot_load(a, slr, xrows + (size_t)sidx * XS, sidx, cnew);
                        if (!xchg && cnew >= 0) {
                            // a lone CTA copies the whole table here, beside the
                            // other warps' slot work (with a cluster, each member
                            // copies its own range after the exchange, below)
                            copy_k_range<16>(a, grp, sidx, cnew, 0, 8 * n_blk, lane, 32);
                            fence_proxy_global();
                            __syncwarp();
                            if (lane == 0) slr.kcell = cnew;
                        }
                        // their K tables and states into L2 ahead of their
                        // refills (whichever slots take them), so that those
                        // wait on L2 rather than DRAM
#pragma unroll
                        for (int d = 0; d < 2; d++)
                            if (cn[d] >= 0) {
                                const uint32_t n_ch = (uint32_t)a.t.n_blk * 8u;
                                if (lane == 0) bulk_prefetch_l2(a.K32 + (size_t)cn[d] * n_ch, n_ch * 16u);
                                if (lane * 16 < N) prefetch_l2(a.rho + (size_t)cn[d] * N + lane * 16);
                            }
                    } else if (lane == 0) {
                        slr = loc;
                    }
                    __syncwarp();
                }
                if (xchg) {
                    // the slot's stage input (16-byte pieces; the row is 16-byte
                    // aligned and zero past N) and cell, to every other CTA
                    const float4 *xs = (const float4 *)(xrows + (size_t)sidx * XS);
                    const uint32_t xoff = (uint32_t)((size_t)sidx * XS * 4);
                    const uint32_t coff = (uint32_t)((size_t)sidx * sizeof(Slot) + offsetof(Slot, cell));
                    const int cell_now = slr.cell;
                    const int n4 = (N + 3) / 4;
                    const float4 xv = lane < n4 ? xs[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 xw = lane + 32 < n4 ? xs[lane + 32] : make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int o = 0; o < P; o++) {
                        if (o == rank) continue;
                        const uint32_t xdst = mapa(su32(xrows), member(o)) + xoff;
                        if (lane < n4) st_cluster_v4(xdst + 16 * lane, xv.x, xv.y, xv.z, xv.w);
                        if (lane + 32 < n4) st_cluster_v4(xdst + 16 * (lane + 32), xw.x, xw.y, xw.z, xw.w);
                        if (lane == 0) st_cluster_s32(mapa(su32(slots), member(o)) + coff, cell_now);
                    }
                }
            }
            if (xchg) {
                fence_cluster();
                __syncwarp();
                if (lane == 0)
                    for (int o = 0; o < P; o++)
                        if (o != rank) mbar_arrive_remote(mapa(su32(xg_full), member(o)));
                if (!cwait(xg_full, r & 1, &s_err, ERR_WAIT_PEER)) break;
            }
            // generic-proxy writes to the stage memory (D staging) must be
            // ordered before the bulk copies of the next pass overwrite it
            fence_async_smem();
            if (!gen_sync(gbar, gphase, &s_err)) break;
            {
                // the slots that took a new cell this pass (refilled here or
                // by another member): this CTA copies its block range of their
                // K tables, all generator threads together, before its
                // producer's next copies read them.  The mask is the same in
                // every warp (all read the slots after the barrier).
                const int ca = slots[lane].cell, cb = slots[lane + 32].cell;
                const unsigned ma = __ballot_sync(0xffffffffu, ca >= 0 && ca != slots[lane].kcell);
                const unsigned mb = __ballot_sync(0xffffffffu, cb >= 0 && cb != slots[lane + 32].kcell);
                const unsigned long long mk = (unsigned long long)ma | ((unsigned long long)mb << 32);
                if (mk) {
                    for (unsigned long long mm = mk; mm; mm &= mm - 1) {
                        const int s2 = __ffsll((long long)mm) - 1;
                        copy_k_range<4>(a, grp, s2, slots[s2].cell, 8 * b_lo, 8 * b_hi, gt, 32 * kGenWarps);
                    }
                    fence_proxy_global();
                    if (!gen_sync(gbar, gphase, &s_err)) break;
                    if (gt == 0)
                        for (unsigned long long mm = mk; mm; mm &= mm - 1) {
                            const int s2 = __ffsll((long long)mm) - 1;
                            slots[s2].kcell = slots[s2].cell;
                        }
                }
            }
            if (gt == 0) {
                int any = 0;
                for (int s2 = 0; s2 < NS; s2++) any |= (slots[s2].cell >= 0);
                if (pairm) {
                    // the pair's MMAs serve both its groups: passes go on while
                    // either has cells (the partner CTA is in the other group)
                    const uint32_t prt = (uint32_t)(crank ^ 1);
                    st_cluster_s32(mapa(su32(&s_any_x), prt), any);
                    fence_cluster();
                    mbar_arrive_remote(mapa(su32(cx_full), prt));
                    if (twait_cluster(cx_full, r & 1, &s_err, ERR_WAIT_PEER)) any |= *(volatile int *)&s_any_x;
                    else any = 0;
                }
                s_continue = any;
                mbar_arrive(go);
            }
            if (!gen_sync(gbar, gphase, &s_err)) break;
            if (!s_continue) break;
        }
    }
    if (warp == 1 && lane == 0) {
        // every MMA this thread (pair mode: the even CTA's) issued has completed
        // before TMEM is freed
        if constexpr (!Pair) mma_commit(fin);
        else if (leader) mma_commit2(fin, pair_mask);
        mbar_drain(fin, 0);
    }
    tc_fence_before();
    if (pairm) cluster_sync_all();                    // neither CTA of a pair frees TMEM before both are done
    else __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        if constexpr (Pair)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
    if (threadIdx.x == 0 && s_err) atomicCAS(a.err, 0, s_err);
    // no CTA of a cluster leaves while another may still write to it
    if (clustered) cluster_sync_all();
}

struct Config { int grid, groups, P, NS, XS, SB, KS, NBP, nacc, stacked, C, sst_off, pair; size_t smem; bool ok; };

cudaError_t launch_kernel(const Config &cf, const MixedArgs &a, cudaStream_t stream);
int sm_count();

// Clusters of P CTAs that can run at once (the launch's groups must all be
// resident together: a group that started late would find its initial cells
// untouched).  Asked of the runtime once per device, P and shared-memory size.
// The kernel instance of a launch: CTA pairs or single CTAs, and the bins per
// lane of the per-slot logic (4 up to 128 bins; CTA pairs need <= 128).  The
// instances share their static shared memory and launch shape.
using MixedKernel = void (*)(MixedArgs);
MixedKernel mixed_kernel(bool pair, int N)
{
    if (pair) return step_mixed_kernel<true, 4>;
    return N <= 128 ? step_mixed_kernel<false, 4> : step_mixed_kernel<false, kLaneBins>;
}

int max_clusters(int P, size_t smem, int n_sm, bool pair = false)   // P: the cluster size
{
    if (P == 1) return n_sm;
    struct Entry { int dev, P; size_t smem; int n; };
    static std::mutex mu;
    static Entry cache[32];
    static int n_cache = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < n_cache; i++)
        if (cache[i].dev == dev && cache[i].P == (pair ? -P : P) && cache[i].smem == smem) return cache[i].n;
    int n = 0;
    auto kern = mixed_kernel(pair, pair ? 128 : kMaxMixedBins);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)(P * (n_sm / P)));
        lc.blockDim = dim3(kThreads);
        lc.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)P;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(&n, kern, &lc);
    }
    if (e != cudaSuccess) {
        n = 0;
        cudaGetLastError();   // clear the error of the refused query (the caller takes a smaller P)
    }
    n = std::min(n, n_sm / P);
    if (n_cache < 32) cache[n_cache++] = {dev, pair ? -P : P, smem, n};
    return n;
}

// Launch layout for clusters of P CTAs (ok = false when P does not fit: fewer
// than two mapping-tile stages beside the buffers, fewer than two stages of a
// pass per CTA, or no cluster of P resident).
// pair: CTA pairs share M = 256 MMAs, a cluster of 2 P CTAs serving two
// groups of 64 slots (each CTA keeps half of every mapping tile)
// Static shared memory of the kernel (as compiled; 2048 if the runtime cannot
// say), asked once per instantiation.
size_t static_smem_bytes(bool pair)
{
    static size_t cached[2] = {0, 0};
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    size_t &v = cached[pair ? 1 : 0];
    if (v == 0) {
        cudaFuncAttributes fa;
        const cudaError_t e = cudaFuncGetAttributes(&fa, mixed_kernel(pair, pair ? 128 : kMaxMixedBins));
        v = (e == cudaSuccess && fa.sharedSizeBytes > 0 && fa.sharedSizeBytes <= 8192) ? fa.sharedSizeBytes : 2048;
        if (e != cudaSuccess) cudaGetLastError();
    }
    return v;
}

// sb_req, ks_req > 0: exactly that many mapping-tile / K-table stages (the
// per-slot state then takes shared memory only if it still fits); 0: the
// automatic choice below.
Config config_for(int n_cells, int N, int P, int n_sm, bool pair = false, int sb_req = 0,
                  int ks_req = 0)   // n_sm: the SMs this launch may occupy
{
    Config c;
    c.P = P;
    c.pair = pair ? 1 : 0;
    const int Q = pair ? 2 * P : P;              // CTAs per cluster
    c.NS = kSlots;
    const int n16 = ((N + 15) / 16) * 16;
    c.XS = n16 + 4;                              // rows 16 B aligned, 4 words off the bank period
    c.NBP = mixed_nbp(N);                        // (the generators read x up to index n16 - 1)
    // TMEM: 512 columns = generated stages + (nacc + 1) accumulators of NBP,
    // or stacked (MMA N = 2 NBP at most 256) nacc accumulators of 2 NBP
    c.stacked = 2 * c.NBP <= 256 ? 1 : 0;
    c.nacc = c.stacked ? std::max(1, std::min(kMaxMain, (512 - kAStages * 64) / (2 * c.NBP)))
                       : std::max(1, std::min(kMaxMain, (512 - kAStages * 64) / c.NBP - 1));
    int n_blk = 0;
    for (int i = 0; i < N; i++) n_blk += (i + kBlkPairs) / kBlkPairs;
    const int n_st = (n_blk + 1) / 2;
    // a stage: two blocks of tiles (pair mode: this CTA's half of each)
    const size_t sstride = 2 * ((((pair ? 1 : 2) * (size_t)c.NBP * 128 + 1023) / 1024) * 1024);
    const int max_sb = pair ? kMaxSB : 4;
    const size_t tail = (size_t)kSlots * c.XS * 4 + (size_t)kSlots * sizeof(Slot) +
                        8 * (3 * kMaxSB + 2 * kAStages + 7 + 2 * kMaxKS + kGenWarps / 2);
    // opt-in shared memory less the kernel's static shared memory and the
    // 1024-byte alignment of the dynamic base
    const size_t budget = 232448 - 1024 - static_smem_bytes(pair);
    const int SL = kSlots / P;
    const size_t dpeer = (size_t)(P - 1) * SL * c.NBP * 4;   // partial sums from the other CTAs
    const size_t room = budget > tail + dpeer ? budget - tail - dpeer : 0;
    // the rings and the per-slot state: the fewest mapping-tile stages that
    // overlap (two, one for a single CTA that fits no more), two K-table
    // stages (they come from DRAM), then the per-slot state if it fits (its
    // per-step reads and writes stay on chip), then more K and tile stages
    const size_t kstage = 2 * (size_t)kKBlkBytes;
    const size_t state = (size_t)SL * 5 * N * sizeof(float);
    const int sb_min = P > 1 ? 2 : (room >= 2 * sstride + kstage ? 2 : 1);
    int SB, KS;
    bool st_smem;
    if (sb_req > 0 || ks_req > 0) {
        SB = sb_req > 0 ? sb_req : sb_min;
        KS = ks_req > 0 ? ks_req : 2;
        const size_t rings = (size_t)SB * sstride + (size_t)KS * kstage;
        st_smem = rings + state <= room;
    } else {
        size_t avail = room > sb_min * sstride ? room - sb_min * sstride : 0;
        KS = (int)std::min<size_t>(2, avail / kstage);
        avail -= KS * kstage;
        st_smem = KS >= 2 && avail >= state;
        if (st_smem) avail -= state;
        const int KSx = (int)std::min<size_t>(kMaxKS - KS, avail / kstage);
        KS += KSx;
        avail -= KSx * kstage;
        SB = sb_min + (int)std::min<size_t>(max_sb - sb_min, avail / sstride);
        // the D staging areas ([slots kept + 64][NBP] floats) alias the mapping-tile ring
        while ((size_t)SB * sstride < (size_t)(SL + kSlots) * c.NBP * 4 && SB < max_sb) SB++;
    }
    c.SB = SB;
    c.KS = KS;
    c.sst_off = st_smem ? (int)((size_t)SB * sstride + KS * kstage) : -1;
    const size_t used = (size_t)SB * sstride + KS * kstage + (st_smem ? state : 0);
    // at least 120 KB, so that no two CTAs share an SM (each holds all 512
    // TMEM columns for the whole kernel)
    c.smem = std::max((size_t)120 * 1024, 1024 + used + tail + dpeer);
    c.ok = KS >= 1 && KS <= kMaxKS && SB >= (P > 1 ? 2 : 1) && SB <= max_sb && used <= room &&
           (P == 1 || n_st >= 2 * P) && (size_t)SB * sstride >= (size_t)(SL + kSlots) * c.NBP * 4 &&
           (!pair || c.stacked);
    // cells are spread over up to one cluster per Q SMs, at least 8 a group
    const int mc = Q == 1 ? n_sm : (c.ok ? std::min(max_clusters(Q, c.smem, sm_count(), pair), n_sm / Q) : 0);
    if (mc < 1) c.ok = false;
    if (pair) {
        const int clusters = std::max(1, std::min(std::max(mc, 1), (n_cells + 15) / 16));
        c.groups = 2 * clusters;
        c.grid = Q * clusters;
    } else {
        c.groups = std::max(1, std::min(std::max(mc, 1), (n_cells + 7) / 8));
        c.grid = P * c.groups;
    }
    c.C = std::min(kSlots, (n_cells + c.groups - 1) / c.groups);
    return c;
}

int sm_count()
{
    int dev = 0, n_sm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    return n_sm;
}

// The cluster size for a request (0: automatic).  Automatic takes the P of
// least modelled time: a pass costs about (1/P + 0.05) of a one-CTA pass (the
// tensor work and per-slot logic divide by P, the exchanges do not), and the
// passes a group runs are about max(1, n_cells / (3 slots)), the costliest
// cells taking about three times the mean.  A request that does not fit
// falls back to the largest smaller P that does.
// max_sms > 0: the launch may occupy at most that many SMs.
// pair_req: 2 = CTA pairs (P_req pairs per cluster, 0: two), falling back to
// fewer pairs and then to single CTAs when it does not fit; otherwise single
// CTAs as below.  sb_req, ks_req: ring depths (0: automatic), see config_for;
// the result's ok is false when no P takes them.
Config mixed_config(int n_cells, int N, int P_req, int max_sms, int pair_req = 0, int sb_req = 0, int ks_req = 0)
{
    const int n_sm = max_sms > 0 ? std::min(max_sms, sm_count()) : sm_count();
    if (pair_req == 2) {
        for (int P = P_req > 0 ? P_req : 2; P >= 1; P /= 2) {
            Config c = config_for(n_cells, N, P, n_sm, true, sb_req, ks_req);
            if (c.ok) return c;
        }
        P_req = 0;
    }
    if (P_req > 0) {
        for (int P = P_req; P >= 1; P /= 2) {
            Config c = config_for(n_cells, N, P, n_sm, false, sb_req, ks_req);
            if (c.ok || P == 1) return c;
        }
    }
    Config best = config_for(n_cells, N, 1, n_sm, false, sb_req, ks_req);
    double best_cost = 1e300;
    for (int P = 1; P <= 8; P *= 2) {
        Config c = config_for(n_cells, N, P, n_sm, false, sb_req, ks_req);
        if (!c.ok) continue;                    // (P = 1 stays the answer when nothing fits)
        const double slots = (double)c.groups * kSlots;
        const double cost = std::max(1.0, n_cells / (3.0 * slots)) * (1.0 / P + 0.05);
        if (cost < best_cost) { best_cost = cost; best = c; }
    }
    return best;
}

cudaError_t launch_kernel(const Config &cf, const MixedArgs &a, cudaStream_t stream)
{
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cf.grid);
    lc.blockDim = dim3(kThreads);
    lc.dynamicSmemBytes = cf.smem;
    lc.stream = stream;
    cudaLaunchAttribute at[1];
    const int Q = cf.pair ? 2 * cf.P : cf.P;
    if (Q > 1) {
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)Q;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&lc, mixed_kernel(cf.pair != 0, a.t.N), a);
}

// L2 prefetch of the K tables pays when the slot groups' tables (8 KB per
// block and group) do not fit in L2: measured +15 % at 148 groups x 780
// blocks (946 MB), -3.5 % at 33 groups x 364 blocks (98 MB of a 126 MB L2)
int prefetch_k_stages(const Config &cf, int n_blk)
{
    static int l2 = -1;
    if (l2 < 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
            cudaGetLastError();
            v = 0;
        }
        l2 = v;
    }
    const double kbytes = (double)cf.groups * n_blk * kKBlkBytes;
    return (l2 > 0 && kbytes > (double)l2) ? kPrefetchK : 0;
}

cudaError_t launch_mixed(const cudisc_coag_ctx *c, int mode, double *rho, double *drho, double t_span,
                         double *dt_cell, const double *replay_h, const long long *replay_n,
                         long long replay_stride, WorkList wl = WorkList())
{
    Config cf = mixed_config(c->n_cells, c->N, c->mix_P, c->p.max_sms, c->mix_pair ? 2 : 1, c->p.mixed_tile_stages,
                             c->p.mixed_k_stages);
    const size_t need = (size_t)cf.groups * cf.NS * 5 * (size_t)c->N * sizeof(float);
    if (need > c->work_bytes) return cudaErrorInvalidValue;
    if (cf.P != c->mix_P || cf.groups != c->mix_G || cf.C != c->mix_C || cf.pair != c->mix_pair)
        return cudaErrorInvalidValue;   // layout of the K tables
    cudaError_t e = cudaFuncSetAttribute(mixed_kernel(cf.pair != 0, c->N),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cf.smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(c->d_counter + 1, 0, 2 * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    MixedArgs a;
    a.t = c->tables();
    a.K32 = reinterpret_cast<const float4 *>(c->d_K32);
    a.Kslot = c->d_Kslot;
    a.rho = rho;
    a.drho = drho;
    a.t_span = t_span;
    a.dt_cell = dt_cell;
    a.rtol = c->p.rtol;
    a.rtol_f = (float)c->p.rtol;
    a.atol_rel = c->p.atol_rel;
    a.max_steps = c->p.max_substeps;
    a.replay_h = replay_h;
    a.replay_n = replay_n;
    a.replay_stride = replay_stride;
    a.out = c->d_out;
    a.err = c->d_counter + 1;
    a.queue = c->d_counter + 2;
    a.work = (float *)c->d_work;
    a.rec_dt = mode == MODE_STEP ? c->rec_dt : nullptr;
    a.rec_cap = c->rec_cap;
    a.rec_n = mode == MODE_RHS ? nullptr : c->rec_n;
    a.rec_status = mode == MODE_RHS ? nullptr : c->rec_status;
    a.NS = cf.NS;
    a.XS = cf.XS;
    a.SB = cf.SB;
    a.NBP = cf.NBP;
    a.nacc = cf.nacc;
    a.stacked = cf.stacked;
    a.kC = c->mix_C;
    a.KS = cf.KS;
    a.sst_off = cf.sst_off;
    a.P = cf.P;
    a.pair = cf.pair;
    a.wait_cycles = c->inject_wait_cycles > 0 ? c->inject_wait_cycles : kWaitCycles;
    a.withhold = c->inject_withhold;
    a.prefetch_k = prefetch_k_stages(cf, c->n_blk);
    a.wl = wl;
    a.mode = mode;
    return launch_kernel(cf, a, c->stream);
}

} // namespace

// ---- fixed-scratch variant -------------------------------------------------
// Scratch for cudisc_coag_step_static_scratch: the per-slot FP32 integrator
// state (state pair and stage right-hand sides) that the regular entry point
// keeps in the context's workspace whenever it does not fit in shared memory.
// It is a file-scope device array of fixed size, so every GPU that loads this
// library holds these 16 MiB until the process exits.  Host code must not
// pass the symbol itself to a kernel (on the host it only names a stand-in);
// the device address comes from cudaGetSymbolAddress, taken with the
// context's device current at the context's first call of the entry point.
namespace {
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
} // namespace

size_t static_scratch_bytes() { return kStaticScratchBytes; }

size_t mixed_scratch_bytes(int n_cells, int N, int P, int max_sms, int pair, int sb_req, int ks_req)
{
    const Config cf = mixed_config(n_cells, N, P, max_sms, pair ? 2 : 1, sb_req, ks_req);
    return cf.sst_off >= 0 ? 0 : (size_t)cf.groups * cf.NS * 5 * (size_t)N * sizeof(float);
}

cudaError_t launch_step_mixed_static(cudisc_coag_ctx *c, double *rho, double t_span, double *dt_cell,
                                     bool *too_big)
{
    *too_big = false;
    Config cf = mixed_config(c->n_cells, c->N, c->mix_P, c->p.max_sms, c->mix_pair ? 2 : 1, c->p.mixed_tile_stages,
                             c->p.mixed_k_stages);
    // the array is only touched when the per-slot state does not fit in
    // shared memory
    const size_t need = cf.sst_off >= 0 ? 0 : (size_t)cf.groups * cf.NS * 5 * (size_t)c->N * sizeof(float);
    if (need > kStaticScratchBytes) { *too_big = true; return cudaSuccess; }
    if (cf.P != c->mix_P || cf.groups != c->mix_G || cf.C != c->mix_C || cf.pair != c->mix_pair)
        return cudaErrorInvalidValue;   // layout of the K tables
    if (!c->static_scratch) {
        // set-up, once per context, with its device current: the array's
        // device address (a context made after a device reset looks it up
        // again; the old contexts' buffers are gone with that reset anyway)
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return e;
        c->static_scratch = ptr;
    }
    cudaError_t e = cudaFuncSetAttribute(mixed_kernel(cf.pair != 0, c->N),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cf.smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(c->d_counter + 1, 0, 2 * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    MixedArgs a;
    a.t = c->tables();
    a.K32 = reinterpret_cast<const float4 *>(c->d_K32);
    a.Kslot = c->d_Kslot;
    a.rho = rho;
    a.drho = nullptr;
    a.t_span = t_span;
    a.dt_cell = dt_cell;
    a.rtol = c->p.rtol;
    a.rtol_f = (float)c->p.rtol;
    a.atol_rel = c->p.atol_rel;
    a.max_steps = c->p.max_substeps;
    a.replay_h = nullptr;
    a.replay_n = nullptr;
    a.replay_stride = 0;
    a.out = c->d_out;
    a.err = c->d_counter + 1;
    a.queue = c->d_counter + 2;
    a.work = (float *)c->static_scratch;   // every slot's state is written before it is read
    a.rec_dt = c->rec_dt;
    a.rec_cap = c->rec_cap;
    a.rec_n = c->rec_n;
    a.rec_status = c->rec_status;
    a.NS = cf.NS;
    a.XS = cf.XS;
    a.SB = cf.SB;
    a.NBP = cf.NBP;
    a.nacc = cf.nacc;
    a.stacked = cf.stacked;
    a.kC = c->mix_C;
    a.KS = cf.KS;
    a.sst_off = cf.sst_off;
    a.P = cf.P;
    a.pair = cf.pair;
    a.wait_cycles = c->inject_wait_cycles > 0 ? c->inject_wait_cycles : kWaitCycles;
    a.withhold = c->inject_withhold;
    a.prefetch_k = prefetch_k_stages(cf, c->n_blk);
    a.wl = WorkList();
    a.mode = MODE_STEP;
    return launch_kernel(cf, a, c->stream);
}

bool mixed_layout(int n_cells, int N, int P_req, int max_sms, int pair_req, int sb_req, int ks_req, int *P, int *G,
                  int *C, int *pair)
{
    const Config cf = mixed_config(n_cells, N, P_req, max_sms, pair_req, sb_req, ks_req);
    *P = cf.P;
    *G = cf.groups;
    *C = cf.C;
    *pair = cf.pair;
    return cf.ok;
}

void mixed_rings(int n_cells, int N, int P, int max_sms, int pair, int sb_req, int ks_req, int *SB, int *KS,
                 int *state_smem)
{
    const Config cf = mixed_config(n_cells, N, P, max_sms, pair ? 2 : 1, sb_req, ks_req);
    *SB = cf.SB;
    *KS = cf.KS;
    *state_smem = cf.sst_off >= 0 ? 1 : 0;
}

size_t mixed_workspace_bytes(int n_cells, int N, int P, int max_sms, int pair, int sb_req, int ks_req)
{
    Config cf = mixed_config(n_cells, N, P, max_sms, pair ? 2 : 1, sb_req, ks_req);
    return (size_t)cf.groups * cf.NS * 5 * (size_t)N * sizeof(float);
}

cudaError_t launch_rhs_mixed(const cudisc_coag_ctx *c, const double *rho, double *drho)
{
    return launch_mixed(c, MODE_RHS, const_cast<double *>(rho), drho, 1.0, nullptr, nullptr, nullptr, 0);
}

cudaError_t launch_step_mixed(const cudisc_coag_ctx *c, double *rho, double t_span, double *dt_cell,
                              const double *replay_h, const long long *replay_n, long long replay_stride,
                              WorkList wl)
{
    return launch_mixed(c, replay_h ? MODE_REPLAY : MODE_STEP, rho, nullptr, t_span, dt_cell, replay_h,
                        replay_n, replay_stride, wl);
}

} // namespace cdc
