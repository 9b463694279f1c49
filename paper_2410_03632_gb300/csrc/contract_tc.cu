// Tensor-core contraction (a) with the R-sum of quadrature (b) fused into the
// epilogue, for a batch of cosmologies:
//
//   w_b(t, l, q) = sum_n a_b[n] T~[t][l][n][q]                       (Eq. pmd)
//   Y_b(t, l, a, rt, j) = sum_{r in R-tile rt} V_bj(a, r) w_b(t, l, a n_R + r)
//
// as one GEMM per (t, l): M = cosmologies (128 per CTA, TMEM lanes), N = 32
// chi-R nodes (one R-tile), K = Chebyshev order (<= 96).  The expansion of P
// in Chebyshev polynomials cancels strongly where P is small (high l, low-z
// lensing), so an FP32-accumulated hi/lo split is not accurate enough.
// Instead both operands are cut into S = 5 fixed-point slices of 8 bits:
//
//   a_b[n]     = 2^ea(b)    sum_p 2^(-8(p+1)) A_p[b][n],   A_p integers, |A_p| <= 256
//   T~[.][n][q] = 2^eT(col) sum_p 2^(-8(p+1)) T_p[col][n]
//
// Slice p is stored as A_p 2^(-8p) (T_q 2^(-8q)): an integer of at most 9
// bits times a power of two, exact in BF16.  Every product is exact, and level
// k, D_k 2^(-8k) = sum_{p+q=k} sum_n (A_p 2^-8p)(T_q 2^-8q), is a multiple of
// 2^(-8k) below 2^(24-8k) in magnitude for K <= 96, so the FP32 tensor-core
// accumulation of levels 0, 1 and 2 is exact.  The 15 slice pairs p+q <= 4
// feed five level accumulators in TMEM (two buffers of 5 x 32 columns).  For
// K <= 64 all five coefficient slices sit in TMEM beside them; for K <= 96
// (two 64-wide K chunks) slices 0..3 do and slice 4, used by one slice pair
// per K step, is read from shared memory.  The epilogue combines the levels with two
// exact fast two-sums and one plain sum of the small parts,
//   W 2^-32 = m + lo,   m = fl(fl(D_0 + D_1) + D_2),   lo = (e_1 + e_2) + (D_3 + D_4),
// and scales by 2^(ea + eT - 16).  The R sum that follows also cancels (w
// oscillates around R = 1), so it runs on unevaluated pairs: exact products
// (FMA), two products (columns two R nodes apart) added plainly, and two-sum
// accumulation of those sums, two columns at a time in packed FP32 pairs; the
// pairs reach the chi sum intact.
//
// Warp roles (320 threads): warp 0 issues TMA loads of the basis slices into
// a ring of stages, warp 1 owns TMEM and issues tcgen05.mma (A = coefficient
// slices resident in TMEM, B = basis slices in shared memory) into two
// accumulator buffers, warps 2..9 run the epilogue (one TMEM lane = one
// cosmology per thread, two warps per lane quadrant with 16 columns each,
// quadrature weights of the unit's five B-side tracers in registers, the two
// column halves joined through shared memory at a named barrier).  A work unit
// is (cosmology tile of 128, group of five B-side tracers, 32-node q tile);
// plans with up to ten tracers per kind run two groups as separate units.
// Every mbarrier wait is bounded; on timeout the kernel records an error code
// in host-mapped memory and exits after its copies and MMAs in flight complete.
#include <cuda.h>
#include <cuda_bf16.h>

#include <climits>
#include <cmath>
#include <cstring>

#include "blast_internal.h"

namespace {

constexpr int kS = BLAST_TC_SLICES;       // slices per operand
constexpr int kQT = 32;                   // chi-R nodes per tile (MMA N)
constexpr int kM = 128;                   // cosmologies per tile (MMA M)
constexpr int kKC = 64;                   // K elements per 128-byte swizzle row (one TMA box)
constexpr int kEP = 2;                    // epilogue warps per TMEM lane quadrant
constexpr int kThreads = 64 + 128 * kEP;  // 2 control warps + 4 kEP epilogue warps
constexpr int kHC = kQT / kEP;            // columns per epilogue thread
constexpr int kCS = 4;                    // columns per TMEM load step
constexpr int kNB = 5;                    // tracers per weight group
constexpr int kNBUF = 2;                  // TMEM accumulator buffers
constexpr uint32_t kBSliceBytes = kQT * 128;  // 32 rows x 64 bf16
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kCtrlBytes = 256;          // mbarriers, TMEM address, abort flag
constexpr uint32_t kEselBytes = 4 * BLAST_MAX_ELL;  // selected ells
constexpr long long kWaitLimit = 4000000000LL;  // clock cycles (about 2 s)
constexpr uint32_t kSuspendNs = 1000000;        // longest suspension of one phase test

// Compile-time shape of one kernel instance: KC 64-wide K chunks per stage
// (1: order <= 64, 2: order <= 96).
// Both keep five exact TMEM levels; with two K chunks the coefficient slices
// 0..3 fill the TMEM left beside the accumulators and slice 4 (one slice pair,
// p = 4, q = 0, per K step) is read from shared memory.
template <int KC> struct TcCfg {
    static constexpr int LV = 5;                            // TMEM accumulator levels
    static constexpr int kStages = KC == 1 ? 8 : 4;
    static constexpr uint32_t kStageBytes = KC * kS * kBSliceBytes;
    static constexpr uint32_t kACol = kNBUF * LV * kQT;     // TMEM column of the coefficient slices
    static constexpr int kSliceTmem = KC == 1 ? kS : kS - 1;  // coefficient slices held in TMEM
    static constexpr uint32_t kA4Bytes = KC == 1 ? 0 : KC * kM * 128;  // slice 4: [chunk][128 rows][128 B]
    static constexpr int kYbufFloats = 2 * 4 * (kEP - 1) * kNB * 64;  // [parity][quadrant][part-1][tracer][hi, lo][lane]
    static constexpr size_t kSmem = 1024 + (size_t)kStages * kStageBytes + kA4Bytes + kCtrlBytes + kEselBytes +
                                    kYbufFloats * 4;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One test of a phase; a thread that finds it incomplete is suspended until the
// phase completes or about kSuspendNs nanoseconds pass, so waiting warps do not
// take issue slots from working ones.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// Barrier among n threads (whole warps) of the CTA on hardware barrier id (1..15).
__device__ __forceinline__ void named_bar_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Bounded wait on a phase: false if it did not complete within kWaitLimit
// cycles.  With sleep_ns > 0 the thread sleeps between tests, doubling up to
// 1 us: for the TMA and MMA warps, which wait most of the time and need not
// answer within a few cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned sleep_ns = 0,
                                          long long limit = kWaitLimit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
        if (sleep_ns) {
            __nanosleep(sleep_ns);
            sleep_ns = min(2u * sleep_ns, 1024u);
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused with 128B swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 128, N = 32.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kQT >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);

// MMA with A read from tensor memory (kM lanes x 16 BF16 packed in 8 columns)
// and B from shared memory; D += A B when acc != 0, D = A B otherwise.
__device__ __forceinline__ void umma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bd, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
        ::"r"(d_tmem), "r"(a_tmem), "l"(bd), "r"(kIdesc), "r"(acc));
}

// MMA with both operands in shared memory (A: kM rows x 16 BF16, K-major).
__device__ __forceinline__ void umma_ss(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d_tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
}

// True in exactly one lane of the (converged) warp.
__device__ __forceinline__ bool elect_one()
{
    uint32_t p;
    asm volatile("{\n\t.reg .pred P;\n\telect.sync _|P, 0xffffffff;\n\tselp.u32 %0, 1, 0, P;\n\t}\n" : "=r"(p));
    return p != 0;
}

// Eight consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld4(uint32_t (&r)[4])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]) : : "memory");
}

// Register fence for values a tcgen05.wait::ld has already covered: ties
// them to a point after that wait.
__device__ __forceinline__ void reg_fence4(uint32_t (&r)[4])
{
    asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]) : : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// Knuth's two-sum: s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    const float ss = __fadd_rn(a, b);
    const float bb = __fsub_rn(ss, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(ss, bb)), __fsub_rn(b, bb));
    s = ss;
}

// Packed pairs of FP32: lane x in the low and lane y in the high half of one
// 64-bit register pair, one instruction for both lanes, rounded to nearest
// like the scalar forms.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float x, float y)
{
    f32x2 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(x), "f"(y));
    return d;
}

__device__ __forceinline__ float2 unpk2(f32x2 a)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a));
    return r;
}

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Both lanes negated (sign bits flipped, exact).
__device__ __forceinline__ f32x2 neg2(f32x2 a) { return a ^ 0x8000000080000000ull; }

// Fast two-sum on both lanes: s + e == a + b exactly when |a| >= |b|, or when
// a + b is representable.
__device__ __forceinline__ void fast_two_sum2(f32x2 a, f32x2 b, f32x2 &s, f32x2 &e)
{
    s = add2(a, b);
    e = sub2(b, sub2(s, a));
}

// Two-sum on both lanes: s + e == a + b exactly.
__device__ __forceinline__ void two_sum2(f32x2 a, f32x2 b, f32x2 &s, f32x2 &e)
{
    const f32x2 ss = add2(a, b);
    const f32x2 bb = sub2(ss, a);
    e = add2(sub2(a, sub2(ss, bb)), sub2(b, bb));
    s = ss;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// One-dimensional bulk copy global -> shared (both 16-byte aligned, size a
// multiple of 16) completing on an mbarrier of this CTA.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------- slicing
// x (|x| < 1) -> S slices: integers in [-256, 256] times 2^(-8p) f for slice
// p, f a power of two (2^-126 <= 2^(-8p) f <= 1), each exact in BF16: the
// powers of two only move the exponent.
__device__ __forceinline__ void slice8(double xn, uint16_t (&out)[kS], float f = 1.0f)
{
    double r = xn * 256.0;
    float sc = f;
#pragma unroll
    for (int p = 0; p < kS; p++) {
        double q = rint(r);
        out[p] = __bfloat16_as_ushort(__float2bfloat16_rn(__fmul_rn((float)q, sc)));
        r = (r - q) * 256.0;
        sc *= 0.00390625f;
    }
}

// Coefficient slices, one warp per cosmology: A_p[b][k] (k < Kst, zero past
// the order) and 2^ea(b); also the chi weights U of both tracer kinds as
// (hi, lo) FP32 pairs, laid out for the reduction's bulk copies:
//   U[bt][a][kind][hl][i][lane],  b = 32 bt + lane,  i < MT (zero past the
//   request's tracer count), kind 0 clustering, 1 lensing.
__global__ void k_coef_slices(const ReqDev *__restrict__ reqs, int n, int N, int Kst, int Bpad, uint16_t *A,
                              float *sa, int X, int MT, float *U, const double *__restrict__ env)
{
    const int b = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (b >= Bpad) return;
    const double *a = (b < n) ? reqs[b].a64 : nullptr;
    // a_n / s_n: the basis rows carry s_n (powers of two, so both scalings are exact)
    double mx = 0.0;
    for (int k = lane; k < N; k += 32) mx = fmax(mx, fabs(a ? a[k] / env[k] : 0.0));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
    for (int k = lane; k < Kst; k += 32) {
        uint16_t s[kS];
        slice8((a && k < N) ? ldexp(a[k] / env[k], -e) : 0.0, s);
#pragma unroll
        for (int p = 0; p < kS; p++) A[((size_t)p * Bpad + b) * Kst + k] = s[p];
    }
    if (lane == 0) sa[b] = ldexpf(1.0f, e);
    const int ng = (b < n) ? reqs[b].n_clust : 0, ns = (b < n) ? reqs[b].n_lens : 0;
    const double *Uq = (b < n) ? reqs[b].U64 : nullptr;
    const int bt = b >> 5, bl = b & 31;
    for (int idx = lane; idx < 2 * MT * X; idx += 32) {
        const int kind = idx / (MT * X), i = (idx / X) % MT, a_ = idx % X;
        const int cnt = kind ? ns : ng, row = kind ? ng + i : i;
        const double u = (i < cnt) ? Uq[(size_t)row * X + a_] : 0.0;
        const float uh = (float)u;
        float *dst = U + ((((size_t)bt * X + a_) * 2 + kind) * 2) * MT * 32 + (size_t)i * 32 + bl;
        dst[0] = uh;
        dst[(size_t)MT * 32] = (float)(u - (double)uh);
    }
}

// Basis slices, one warp per tile of kQT columns (t, l, q0..q0+31), a lane per
// column: T_p[col][k] 2^(-8p) 2^(eT(col) - eG) (k < Kst, zero past the order)
// with eG the largest column exponent of the tile, and one scale 2^(eG - 16)
// per tile.  A column keeps its own 40-bit fixed-point precision; the power of
// two moves the exponent only.  Columns more than 2^90 below the tile's
// largest (or in tiles whose scale underflows FP32) are zero: they could not
// change the tile's sum.
__global__ void k_basis_slices(const double *__restrict__ T, int L, int N, int Q, int Kst, uint16_t *Tsl,
                               float *scT, const double *__restrict__ env)
{
    const size_t ncol = (size_t)3 * L * Q;
    const size_t ntile = ncol / kQT;
    const int lane = threadIdx.x & 31;
    for (size_t tile = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; tile < ntile;
         tile += ((size_t)gridDim.x * blockDim.x) / 32) {
        const size_t col = tile * kQT + lane;
        const size_t tl = col / Q, q = col % Q;
        const double *src = T + tl * (size_t)N * Q + q;
        double mx = 0.0;
        for (int k = 0; k < N; k++) mx = fmax(mx, fabs(src[(size_t)k * Q] * env[k]));
        int e = 0;
        if (mx > 0.0) frexp(mx, &e);
        int eG = (mx > 0.0) ? e : INT_MIN;
        for (int o = 16; o; o >>= 1) eG = max(eG, __shfl_xor_sync(0xffffffffu, eG, o));
        const float scf = (eG != INT_MIN) ? (float)ldexp(1.0, eG - 16) : 0.0f;
        const bool keep = mx > 0.0 && scf != 0.0f && e - eG >= -90;
        const float shift = keep ? ldexpf(1.0f, e - eG) : 0.0f;
        for (int k = 0; k < Kst; k++) {
            uint16_t s[kS];
            slice8((k < N && keep) ? ldexp(src[(size_t)k * Q] * env[k], -e) : 0.0, s, shift);
#pragma unroll
            for (int p = 0; p < kS; p++) Tsl[((size_t)p * ncol + col) * Kst + k] = s[p];
        }
        if (lane == 0) scT[tile] = scf;
    }
}

// ---------------------------------------------------------------- main kernel
struct TcArgs {
    const ReqDev *reqs;
    int n, Bpad, nbt, ngr, nqt, n_esel, L, Q, Rn, RT, MT, X, Kst, Kmma;
    int npass, sym;      // passes per q tile (3, or 4 for the symmetrised form)
    const int *esel;
    const float *scT;    // [3][L][Q / kQT] one scale per tile
    const float *sa;     // [Bpad]
    const uint16_t *A;   // [S][Bpad][Kst] coefficient slices
    float *Y;            // [npass][n_esel][X][Bpad/32][ngr][RT][5][hi, lo][32] R-tile partial pairs
    int *err;            // host-mapped error word
    int trip;            // test hook: tile at which CTA 0 waits on a barrier nothing completes (-1 off)
};

// Passes over one q tile: (basis type, kind of the B-side weights, 0 clustering
// 1 lensing).  Split R form: gg (g), gs (s), ss (s).  Symmetrised form (App.
// A, both kernel orders): gg (g), gs with the clustering weights (g) for the
// K^s(chi) K^g(R chi) term, gs (s), ss (s).
__host__ __device__ __forceinline__ int pass_basis(int pass, int sym)
{
    return sym ? (pass == 0 ? 0 : (pass == 3 ? 2 : 1)) : pass;
}
__host__ __device__ __forceinline__ int pass_kind(int pass, int sym) { return sym ? (pass >= 2) : (pass >= 1); }
// kind of the A-side weights U of a pass
__host__ __device__ __forceinline__ int pass_kind_a(int pass, int sym)
{
    return sym ? (pass == 1 || pass == 3) : (pass == 2);
}

// Work units: (cosmology tile, group of five B-side tracers, 32-column q
// tile).  A CTA keeps its cosmology tile (the grid is a multiple of nbt), so
// the coefficient slices stay in TMEM for the whole launch; each unit runs
// the 3 n_esel (type, ell) tiles of its q tile.
__device__ __forceinline__ void unit_decode(const TcArgs &a, int u, int &grp, int &q0)
{
    grp = (u / a.nbt) % a.ngr;
    q0 = (u / (a.nbt * a.ngr)) * kQT;
}

template <int KC>
__global__ void __launch_bounds__(kThreads, 1)
k_contract_tc(const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapA4, TcArgs args)
{
    using C = TcCfg<KC>;
    constexpr int LV = C::LV;
    constexpr int kStages = C::kStages;
    constexpr int NGB = kNB;  // B-side tracers of one unit
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment for the swizzled tiles
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sB = smem;                                         // kStages x KC x kS x 4 KB
    unsigned char *sA4 = sB + (size_t)kStages * C::kStageBytes;        // coefficient slice 4 (order > 64)
    uint64_t *bars = (uint64_t *)(sA4 + C::kA4Bytes);                   // kCtrlBytes of control words
    uint64_t *full = bars, *empty = bars + kStages, *aready = bars + 2 * kStages;
    uint64_t *tfull = aready + 1, *tempty = tfull + kNBUF, *mdone = tempty + kNBUF, *a4ready = mdone + 1;
    uint64_t *never = a4ready + 1;  // no thread ever arrives on it (test hook)
    uint32_t *tmem_slot = (uint32_t *)(never + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    int *s_esel = (int *)((unsigned char *)bars + kCtrlBytes);         // selected ells
    float *ybuf = (float *)((unsigned char *)s_esel + kEselBytes);     // [2][4][kEP-1][NGB][2][32] column-part hand-over

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int btile = blockIdx.x % args.nbt;
    const int n_iter_unit = args.npass * args.n_esel;
    const int n_units = args.nbt * args.ngr * args.nqt;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; i++) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        mbar_init(aready, 128);
        for (int i = 0; i < kNBUF; i++) { mbar_init(&tfull[i], 1); mbar_init(&tempty[i], 128 * kEP); }
        mbar_init(mdone, 1);
        mbar_init(a4ready, 1);
        mbar_init(never, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < args.n_esel; i += blockDim.x) s_esel[i] = args.esel[i];
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer (whole warp waits, one lane issues)
        if (KC == 2) {  // coefficient slice 4 of this CTA's cosmology tile, once
            if (elect_one()) {
                mbar_expect_tx(a4ready, C::kA4Bytes);
#pragma unroll
                for (int c = 0; c < KC; c++) tma_load_2d(sA4 + c * kM * 128, &mapA4, a4ready, c * kKC, btile * kM);
            }
            __syncwarp();
        }
        uint32_t g = 0;
        bool ok = true;
        for (int u = blockIdx.x; ok && u < n_units; u += gridDim.x) {
            int grp, q0;
            unit_decode(args, u, grp, q0);
            for (int it = 0; it < n_iter_unit; it++, g++) {
                const int st = g % kStages;
                const uint32_t ph = (g / kStages) & 1;
                const bool bad = *abort_flag || !mbar_wait(&empty[st], ph ^ 1, 64);
                if (__any_sync(0xffffffffu, bad)) {
                    if (lane == 0) { atomicExch(args.err, 1); *abort_flag = 1; }
                    ok = false;
                    break;
                }
                if (elect_one()) {
                    const int t = pass_basis(it / args.n_esel, args.sym), e = s_esel[it % args.n_esel];
                    const int row = (t * args.L + e) * args.Q + q0;
                    mbar_expect_tx(&full[st], C::kStageBytes);
#pragma unroll
                    for (int c = 0; c < KC; c++)
                        tma_load_3d(sB + (size_t)st * C::kStageBytes + c * kS * kBSliceBytes, &mapB, &full[st],
                                    c * kKC, row, 0);
                }
                __syncwarp();
            }
        }
        // drain: every issued load has landed before the CTA may exit
        for (uint32_t h = (g > (uint32_t)kStages ? g - kStages : 0); h < g; h++)
            mbar_wait(&full[h % kStages], (h / kStages) & 1, 64);
        if (KC == 2) mbar_wait(a4ready, 0, 64);
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (whole warp waits; each MMA is
        // issued by one elected lane of the converged warp)
        bool ok = __all_sync(0xffffffffu, mbar_wait(aready, 0, 64) && (KC == 1 || mbar_wait(a4ready, 0, 64)));
        if (!ok && lane == 0) { atomicExch(args.err, 2); *abort_flag = 1; }  // coefficient slices in TMEM / smem
        tc_fence_after();
        const uint32_t b0 = __shfl_sync(0xffffffffu, smem_u32(sB), 0);  // warp-uniform operands
        const uint32_t tm = __shfl_sync(0xffffffffu, tmem, 0);
        const int nk = args.Kmma / 16;        // K steps of 16
        const uint32_t a4base = __shfl_sync(0xffffffffu, smem_u32(sA4), 0);
        const uint32_t acol = args.Kmma / 2;  // TMEM columns per coefficient slice
        uint32_t g = 0;
        for (int u = blockIdx.x; ok && u < n_units; u += gridDim.x) {
            for (int it = 0; it < n_iter_unit; it++, g++) {
                const int st = g % kStages;
                const uint32_t ph = (g / kStages) & 1;
                const int buf = g % kNBUF;
                const uint32_t tph = (g / kNBUF) & 1;
                const bool bad = *abort_flag || !mbar_wait(&full[st], ph, 64) || !mbar_wait(&tempty[buf], tph ^ 1, 64);
                if (__any_sync(0xffffffffu, bad)) {
                    if (lane == 0) { atomicExch(args.err, 3); *abort_flag = 1; }
                    ok = false;
                    break;
                }
                tc_fence_after();
                // operands: accumulator levels of this buffer, coefficient slices in
                // TMEM, basis slice descriptors offset from this stage's first
                const uint32_t dbase = tm + buf * (LV * kQT);
                const uint64_t bbase = sdesc(b0 + st * C::kStageBytes);
                if (elect_one()) {
                    // Consecutive MMAs into one accumulator wait for each other, so the
                    // issue order interleaves the levels: per K step, rounds r = 0..4 of
                    // the slice pairs (p = r, q = k - r) over levels k = 4 .. 0, so that
                    // an accumulator is hit again only after the other levels had a turn.
                    uint32_t started = 0;  // levels already written in this tile
                    for (int kk = 0; kk < nk; kk++) {
                        const uint32_t koff = (kk >> 2) * (kS * kBSliceBytes) + (kk & 3) * 32;
#pragma unroll
                        for (int r = 0; r < kS; r++) {
#pragma unroll
                            for (int k = kS - 1; k >= r; k--) {
                                const int p = r, q = k - r;
                                const int lev = k < LV - 1 ? k : LV - 1;
                                const uint32_t boff = koff + q * kBSliceBytes;
                                if (p < C::kSliceTmem)
                                    umma_ts(dbase + lev * kQT, tm + C::kACol + p * acol + kk * 8,
                                            bbase + (uint64_t)(boff >> 4), (started >> lev) & 1u);
                                else  // slice 4 from shared memory
                                    umma_ss(dbase + lev * kQT,
                                            sdesc(a4base + (kk >> 2) * (kM * 128)) + (uint64_t)(((kk & 3) * 32) >> 4),
                                            bbase + (uint64_t)(boff >> 4), (started >> lev) & 1u);
                                started |= 1u << lev;
                            }
                        }
                    }
                }
                __syncwarp();
                if (elect_one()) {
                    umma_commit(&empty[st]);
                    umma_commit(&tfull[buf]);
                }
                __syncwarp();
            }
        }
        // every MMA this warp issued has completed before TMEM is released
        if (elect_one()) umma_commit(mdone);
        __syncwarp();
        mbar_wait(mdone, 0, 64);
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue: kEP warps per TMEM lane quadrant;
        // a thread owns one cosmology (TMEM lane) and kHC of the tile's 32 columns.
        const int ew = warp - 2;
        const int quad = warp & 3;   // lanes 32 quad .. 32 quad + 31 are readable by this warp
        const int part = ew >> 2;    // columns [kHC part, kHC part + kHC)
        const int bl_ = quad * 32 + lane;
        const int b = btile * kM + bl_;
        const bool valid = b < args.n;
        // a quadrant whose 32 lanes are all padding (a batch smaller than the
        // tile) only keeps the buffer hand-off in step
        const bool qlive = btile * kM + quad * 32 < args.n;
        const ReqDev *rq = valid ? &args.reqs[b] : nullptr;
        const int ng = valid ? rq->n_clust : 0, ns = valid ? rq->n_lens : 0;
        const float sa = args.sa[b];
        const uint32_t lane_addr = ((uint32_t)(quad * 32)) << 16;
        const int cb = part * kHC;
        const int tid_e = threadIdx.x - 64;  // 0 .. 128 kEP - 1
        if (part == 0) {
            // coefficient slices of cosmology b -> TMEM lane b, columns kACol + (Kmma/2) p ..
            const int acol = args.Kmma / 2;
#pragma unroll 1
            for (int p = 0; p < C::kSliceTmem; p++) {
                const uint4 *src = reinterpret_cast<const uint4 *>(args.A + ((size_t)p * args.Bpad + b) * args.Kst);
#pragma unroll 1
                for (int c8 = 0; c8 < acol / 8; c8++) {
                    const uint4 v0 = __ldg(src + 2 * c8), v1 = __ldg(src + 2 * c8 + 1);
                    const uint32_t r[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                    tmem_st8(tmem + lane_addr + C::kACol + p * acol + c8 * 8, r);
                }
            }
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(aready);
        }
        // Every thread of the quadrant's two warps passes the same number of
        // named barriers; after a wait runs out the warps skip the work but keep
        // the count, so no barrier is left waiting.
        const int bar_id = 1 + quad;
        uint32_t g = 0;
        bool dead = false;
        f32x2 vr[kNB][kHC / 2];  // quadrature weights (times 2^ea) of tracers 0..4 of the B-side kind
        for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
            int grp, q0;
            unit_decode(args, u, grp, q0);
            const int a = q0 / args.Rn, rt = (q0 % args.Rn) / kQT;
            for (int t = 0; t < args.npass; t++) {  // t: pass (the Y index)
                const int kindB = pass_kind(t, args.sym);
                const int offB = kindB ? ng : 0, nB = kindB ? ns : ng;
                if (t == 0 || kindB != pass_kind(t - 1, args.sym)) {
                    // weights of the pass's B-side kind (passes of one kind follow each
                    // other), tracers 5 grp .. 5 grp + 4 of it
#pragma unroll
                    for (int j = 0; j < kNB; j++) {
                        const int jj = kNB * grp + j;
                        const float4 *src =
                            (valid && jj < nB)
                                ? reinterpret_cast<const float4 *>(rq->V32 + (size_t)(offB + jj) * args.Q + q0 + cb)
                                : nullptr;
#pragma unroll
                        for (int c = 0; c < kHC / 4; c++) {
                            const float4 v = src ? src[c] : make_float4(0.f, 0.f, 0.f, 0.f);
                            vr[j][2 * c] = pk2(v.x * sa, v.y * sa);
                            vr[j][2 * c + 1] = pk2(v.z * sa, v.w * sa);
                        }
                    }
                }
                for (int es = 0; es < args.n_esel; es++, g++) {
                    const int buf = g % kNBUF;
                    const uint32_t tph = (g / kNBUF) & 1;
                    // the tile's scale 2^(eG - 16), fetched while the MMA finishes
                    const float tsc =
                        (part == 0) ? args.scT[((size_t)pass_basis(t, args.sym) * args.L + s_esel[es]) * (args.Q / kQT) +
                                               q0 / kQT]
                                    : 0.f;
                    if (!dead) {
                        bool lost = *abort_flag != 0;
                        // test hook: one warp of CTA 0 waits, with a 20M-cycle limit, on a
                        // barrier nothing completes, so the bounded wait runs out
                        if (!lost && (int)g == args.trip && blockIdx.x == 0 && warp == 2 &&
                            !mbar_wait(never, 0, 0, 20000000LL)) {
                            lost = true;
                            atomicExch(args.err, 4);
                            *abort_flag = 1;
                        }
                        if (!lost && !mbar_wait(&tfull[buf], tph)) {
                            lost = true;
                            atomicExch(args.err, 4);
                            *abort_flag = 1;
                        }
                        dead = __any_sync(0xffffffffu, lost);
                    }
                    float Sh[NGB], Sl[NGB];
#pragma unroll
                    for (int j = 0; j < NGB; j++) { Sh[j] = 0.f; Sl[j] = 0.f; }
                    if (!dead && !qlive) mbar_arrive(&tempty[buf]);  // nothing of this buffer is read
                    if (!dead && qlive) {
                        tc_fence_after();
                        const uint32_t tcol = tmem + lane_addr + buf * (LV * kQT) + cb;
                        // R-sum of this thread's columns, two columns per packed lane pair, as
                        // negated unevaluated sums An + Bn: each product V w is split exactly
                        // (FMA), the two products of a lane pair are added plainly, and each
                        // addition of those sums keeps its rounding error (two-sum), so the
                        // sum survives the cancellation of oscillating w
                        f32x2 An[NGB], Bn[NGB];
#pragma unroll
                        for (int s = 0; s < kHC / kCS; s++) {
                            uint32_t D[LV][kCS];
#pragma unroll
                            for (int lev = 0; lev < LV; lev++) tmem_ld4(tcol + lev * kQT + s * kCS, D[lev]);
                            tmem_wait_ld4(D[0]);
#pragma unroll
                            for (int lev = 1; lev < LV; lev++) reg_fence4(D[lev]);
                            if (s + 1 == kHC / kCS) {  // every level of this buffer is in registers: release it
                                tc_fence_before();
                                mbar_arrive(&tempty[buf]);
                            }
                            // levels 0..2 are exact multiples of their quanta, so both fast
                            // two-sums are exact; the small parts add plainly (one rounding)
                            f32x2 m[kCS / 2], lo[kCS / 2];
#pragma unroll
                            for (int h = 0; h < kCS / 2; h++) {
                                f32x2 d[LV];
#pragma unroll
                                for (int lev = 0; lev < LV; lev++)
                                    d[lev] = pk2(__uint_as_float(D[lev][2 * h]), __uint_as_float(D[lev][2 * h + 1]));
                                f32x2 e1, e2;
                                fast_two_sum2(d[0], d[1], m[h], e1);
                                fast_two_sum2(m[h], d[2], m[h], e2);
                                const f32x2 small = (LV == 5) ? add2(d[3], d[LV - 1]) : d[3];
                                lo[h] = add2(add2(e1, e2), small);
                            }
#pragma unroll
                            for (int ch = 0; ch < kCS / 4; ch++) {
                                const int h0 = 2 * ch, h1 = 2 * ch + 1;
                                const f32x2 mn0 = neg2(m[h0]), mn1 = neg2(m[h1]);
                                const bool first = (s == 0 && ch == 0);
#pragma unroll
                                for (int j = 0; j < NGB; j++) {
                                    const int pc = s * (kCS / 2) + h0;  // packed column pair index
                                    const f32x2 v0 = vr[j][pc], v1 = vr[j][pc + 1];
                                    const f32x2 p0 = mul2(v0, mn0), p1 = mul2(v1, mn1);   // -fl(v m)
                                    const f32x2 e0 = fma2(v0, lo[h0], fma2(v0, m[h0], p0));  // v lo + (v m - fl(v m))
                                    const f32x2 e1 = fma2(v1, lo[h1], fma2(v1, m[h1], p1));
                                    const f32x2 ps = add2(p0, p1), pe = add2(e0, e1);
                                    if (first) {  // the sums start here
                                        An[j] = ps;
                                        Bn[j] = neg2(pe);
                                    } else {
                                        f32x2 se;
                                        two_sum2(An[j], ps, An[j], se);
                                        Bn[j] = add2(Bn[j], sub2(se, pe));
                                    }
                                }
                            }
                        }
                        // both lanes into one pair per tracer: S = -(An.x + An.y) - (Bn.x + Bn.y)
#pragma unroll
                        for (int j = 0; j < NGB; j++) {
                            const float2 A2 = unpk2(An[j]), B2 = unpk2(Bn[j]);
                            float h, el;
                            two_sum(A2.x, A2.y, h, el);
                            Sh[j] = -h;
                            Sl[j] = -__fadd_rn(el, __fadd_rn(B2.x, B2.y));
                        }
                    }
                    // the column parts meet: parts 1.. hand their pairs to part 0 through
                    // shared memory, double buffered by iteration
                    float *yq = ybuf + ((size_t)(g & 1) * 4 + quad) * ((kEP - 1) * NGB * 64);
                    if (part > 0) {
                        float *yp = yq + (part - 1) * (NGB * 64);
#pragma unroll
                        for (int j = 0; j < NGB; j++) { yp[j * 64 + lane] = Sh[j]; yp[j * 64 + 32 + lane] = Sl[j]; }
                    }
                    named_bar_sync(bar_id, 32 * kEP);
                    if (part == 0 && !dead) {
#pragma unroll
                        for (int q = 0; q < kEP - 1; q++) {
                            const float *yp = yq + q * (NGB * 64);
#pragma unroll
                            for (int j = 0; j < NGB; j++) {
                                float se;
                                two_sum(Sh[j], yp[j * 64 + lane], Sh[j], se);
                                Sl[j] = __fadd_rn(Sl[j], __fadd_rn(se, yp[j * 64 + 32 + lane]));
                            }
                        }
                        if (valid) {
                            // times the tile's scale (exact); the pair (hi, lo) of tracer j at
                            // Y[t][es][a][b / 32][rt][j][hi, lo][b % 32]: a warp stores 128 bytes
                            float *y = args.Y +
                                       ((((((size_t)t * args.n_esel + es) * args.X + a) * (args.Bpad / 32) + (b >> 5)) *
                                             args.ngr + grp) * args.RT + rt) * (size_t)kNB * 64 + lane;
#pragma unroll
                            for (int j = 0; j < NGB; j++) { y[j * 64] = Sh[j] * tsc; y[j * 64 + 32] = Sl[j] * tsc; }
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// Sum over R tiles and chi nodes for the tensor-core path.  A block handles
// (32 cosmologies, selected ell, type, group of five B-side tracers) and W
// warps split the chi nodes; a thread owns one cosmology and accumulates every
// tracer pair (i, j) of its group, i over all A-side tracers (MTA <= 10):
//   s_j(a) = sum_rt Y(t, l, a, rt, j)          (pairs (hi, lo), two-sum)
//   C_ij(l) = N_AB(l) sum_a U_i(a) s_j(a)      (exact products, two-sum)
// Each warp streams its chi nodes through a ring of NS shared-memory stages:
// one bulk copy brings the 32 cosmologies' R-tile pairs of the group at a chi
// node (contiguous in Y), another their chi weights; the chunks meet in a
// tree through the same shared memory at the end.
//
// Symmetrised form (sym != 0): the block's pass gives one kernel order, every
// pair (i, j) of it, times N_AB(l), is written to S[b][pass][i][j][es], and
// k_sym_combine adds the two orders of each spectrum.
template <int MTA>
__global__ void __launch_bounds__(256)
k_reduce_tc(const ReqDev *__restrict__ reqs, const float *__restrict__ Y, const float *__restrict__ U, int n,
            int X, int L, const int *__restrict__ esel, int n_esel, int RT, int MT, int nbt32, int ngr, int NS,
            const double *__restrict__ pref, int *err, int sym, double *__restrict__ S)
{
    extern __shared__ __align__(128) unsigned char red_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int bt = blockIdx.x, es = blockIdx.y;
    const int t = blockIdx.z / ngr, grp = blockIdx.z % ngr;
    const int b = bt * 32 + lane;
    const ReqDev *rq = (b < n) ? &reqs[b] : nullptr;
    const int ng = rq ? rq->n_clust : 0, ns = rq ? rq->n_lens : 0;
    const int kindA = pass_kind_a(t, sym), kindB = pass_kind(t, sym);  // t: pass
    const int nA = kindA ? ns : ng, nB = kindB ? ns : ng;
    const int e = esel[es];
    const int col = rq ? rq->e_out[e] : -1;
    const int yfl = RT * kNB * 64, ufl = 2 * MT * 32, stf = yfl + ufl;  // floats per stage
    float *ring = reinterpret_cast<float *>(red_smem) + (size_t)w * NS * stf;
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<float *>(red_smem) + (size_t)W * NS * stf) + w * NS;
    if (lane == 0) {
        for (int s = 0; s < NS; s++) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const int per = (X + W - 1) / W;
    const int a0 = w * per, cnt = max(0, min(X, a0 + per) - a0);
    const size_t ystride = (size_t)nbt32 * ngr * yfl;  // floats between chi nodes
    const float *Yb = Y + ((size_t)t * n_esel + es) * (size_t)X * ystride + ((size_t)bt * ngr + grp) * yfl;
    const float *Ub = U + (size_t)bt * X * 2 * ufl + (size_t)kindA * ufl;
    auto issue = [&](int k) {  // chi node a0 + k into stage k % NS
        if (k < cnt && lane == 0) {
            float *d = ring + (size_t)(k % NS) * stf;
            const int a = a0 + k;
            fence_proxy_async();
            mbar_expect_tx(&bars[k % NS], (uint32_t)stf * 4);
            bulk_g2s(d, Yb + (size_t)a * ystride, (uint32_t)yfl * 4, &bars[k % NS]);
            bulk_g2s(d + yfl, Ub + (size_t)a * 2 * ufl, (uint32_t)ufl * 4, &bars[k % NS]);
        }
    };
    for (int k = 0; k < NS; k++) issue(k);
    float Zh[MTA][kNB], Zl[MTA][kNB];
#pragma unroll
    for (int i = 0; i < MTA; i++)
#pragma unroll
        for (int j = 0; j < kNB; j++) { Zh[i][j] = 0.f; Zl[i][j] = 0.f; }
    int done = 0;  // chi nodes whose stage was consumed
    bool aborted = false;
    for (int k = 0; k < cnt; k++, done++) {
        const bool bad = !mbar_wait(&bars[k % NS], (k / NS) & 1);
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0) atomicExch(err, 5);
            aborted = true;
            break;
        }
        const float *v = ring + (size_t)(k % NS) * stf;
        float sv[kNB], sle[kNB];
#pragma unroll
        for (int j = 0; j < kNB; j++) {
            float sh = 0.f, sl = 0.f;
            if (kNB * grp + j < nB) {
#pragma unroll 2
                for (int rt = 0; rt < RT; rt++) {
                    const float yh = v[(rt * kNB + j) * 64 + lane], yl = v[(rt * kNB + j) * 64 + 32 + lane];
                    float se;
                    two_sum(sh, yh, sh, se);
                    sl = __fadd_rn(sl, __fadd_rn(se, yl));
                }
            }
            two_sum(sh, sl, sv[j], sle[j]);
        }
        const float *u = v + yfl;  // [hl][MT][32]
#pragma unroll
        for (int i = 0; i < MTA; i++) {
            if (i >= nA) continue;
            const float uh = u[i * 32 + lane], ul = u[(MT + i) * 32 + lane];
#pragma unroll
            for (int j = 0; j < kNB; j++) {
                const float pr = __fmul_rn(uh, sv[j]);
                const float pe = fmaf(uh, sle[j], fmaf(ul, sv[j], fmaf(uh, sv[j], -pr)));
                float se;
                two_sum(Zh[i][j], pr, Zh[i][j], se);
                Zl[i][j] = __fadd_rn(Zl[i][j], __fadd_rn(se, pe));
            }
        }
        __syncwarp();  // every lane has read the stage before it is refilled
        issue(k + NS);
    }
    // copies still in flight (after a wait gave up) land before the memory is reused
    if (aborted)
        for (int k = done; k < min(cnt, done + NS); k++) mbar_wait(&bars[k % NS], (k / NS) & 1);
    __syncthreads();  // the staging rings become the tree's exchange area
    float *red = reinterpret_cast<float *>(red_smem);  // [W/2][32][2 MTA kNB]
    constexpr int ZP = 2 * MTA * kNB;
    for (int half = W / 2; half >= 1; half >>= 1) {
        if (w >= half && w < 2 * half) {
#pragma unroll
            for (int i = 0; i < MTA; i++)
#pragma unroll
                for (int j = 0; j < kNB; j++) {
                    red[((w - half) * 32 + lane) * ZP + 2 * (i * kNB + j)] = Zh[i][j];
                    red[((w - half) * 32 + lane) * ZP + 2 * (i * kNB + j) + 1] = Zl[i][j];
                }
        }
        __syncthreads();
        if (w < half) {
#pragma unroll
            for (int i = 0; i < MTA; i++)
#pragma unroll
                for (int j = 0; j < kNB; j++) {
                    float se;
                    two_sum(Zh[i][j], red[(w * 32 + lane) * ZP + 2 * (i * kNB + j)], Zh[i][j], se);
                    Zl[i][j] = __fadd_rn(Zl[i][j], __fadd_rn(se, red[(w * 32 + lane) * ZP + 2 * (i * kNB + j) + 1]));
                }
        }
        __syncthreads();
    }
    if (w != 0 || !rq || col < 0) return;
    const double pf = pref[pass_basis(t, sym) * L + e];
    if (sym) {
#pragma unroll
        for (int i = 0; i < MTA; i++) {
#pragma unroll
            for (int j = 0; j < kNB; j++) {
                const int jb = kNB * grp + j;
                if (i >= nA || jb >= nB) continue;
                S[((((size_t)b * 4 + t) * MT + i) * MT + jb) * n_esel + es] = pf * ((double)Zh[i][j] + (double)Zl[i][j]);
            }
        }
        return;
    }
    const int ngg = ng * (ng + 1) / 2, ngs = ng * ns;
#pragma unroll
    for (int i = 0; i < MTA; i++) {
#pragma unroll
        for (int j = 0; j < kNB; j++) {
            const int jb = kNB * grp + j;
            if (i >= nA || jb >= nB) continue;
            int p;
            if (t == 0) { if (i > jb) continue; p = i * ng - i * (i - 1) / 2 + (jb - i); }
            else if (t == 1) p = ngg + i * ns + jb;
            else { if (i > jb) continue; p = ngg + ngs + i * ns - i * (i - 1) / 2 + (jb - i); }
            double out = pf * ((double)Zh[i][j] + (double)Zl[i][j]);
            if (rq->status) out = nan("");
            rq->cl[(size_t)p * rq->n_sel + col] = out;
        }
    }
}

// The symmetrised form's two kernel orders of every spectrum (App. A):
//   gg, ss: C_ij = S[pass][i][j] + S[pass][j][i]   (i <= j; the diagonal doubles)
//   gs:     C_ij = S[gs][i][j] + S[gs with clustering weights][j][i]
// one addition per output, so the result does not depend on the launch.
__global__ void k_sym_combine(const ReqDev *__restrict__ reqs, const double *__restrict__ S, int MT,
                              const int *__restrict__ esel, int n_esel)
{
    const int b = blockIdx.y;
    const ReqDev &rq = reqs[b];
    const int ng = rq.n_clust, ns = rq.n_lens;
    const int ngg = ng * (ng + 1) / 2, ngs = ng * ns, P = ngg + ngs + ns * (ns + 1) / 2;
    const double *Sb = S + (size_t)b * 4 * MT * MT * n_esel;
    auto at = [&](int pass, int i, int j, int es) { return Sb[(((size_t)pass * MT + i) * MT + j) * n_esel + es]; };
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < P * n_esel; idx += gridDim.x * blockDim.x) {
        const int p = idx / n_esel, es = idx % n_esel;
        const int col = rq.e_out[esel[es]];
        if (col < 0) continue;
        double v;
        if (p < ngg || p >= ngg + ngs) {  // gg or ss: (i, j), i <= j, of the pass's kind
            const bool ss = p >= ngg;
            const int m = ss ? ns : ng;
            int i = 0, rem = ss ? p - ngg - ngs : p;
            while (rem >= m - i) { rem -= m - i; i++; }
            const int j = i + rem, pass = ss ? 3 : 0;
            v = at(pass, i, j, es) + at(pass, j, i, es);
        } else {
            const int i = (p - ngg) / ns, j = (p - ngg) % ns;  // clustering i, lensing j
            v = at(2, i, j, es) + at(1, j, i, es);
        }
        if (rq.status) v = nan("");
        rq.cl[(size_t)p * rq.n_sel + col] = v;
    }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    // looked up once; the initialisation of a function-local static is thread safe
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (EncodeTiledFn)p;
        return (EncodeTiledFn) nullptr;
    }();
    return fn;
}

// 2-D map over [rows][Kst] bf16, box {64, box_rows}, 128-byte swizzle.
int make_map2d(CUtensorMap *m, void *base, int Kst, long long rows, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return BLAST_EDEVICE;
    cuuint64_t dims[2] = {(cuuint64_t)Kst, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kst * 2};
    cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        blast_last_error(__FILE__, __LINE__, "cuTensorMapEncodeTiled failed");
        return BLAST_EDEVICE;
    }
    return BLAST_OK;
}

// 3-D map over [S][rows][Kst] bf16, box {64, box_rows, S}, 128-byte swizzle;
// boxes at x = 64 past Kst read zeros.
int make_map(CUtensorMap *m, void *base, int Kst, long long rows, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return BLAST_EDEVICE;
    cuuint64_t dims[3] = {(cuuint64_t)Kst, (cuuint64_t)rows, (cuuint64_t)kS};
    cuuint64_t strides[2] = {(cuuint64_t)Kst * 2, (cuuint64_t)rows * Kst * 2};
    cuuint32_t box[3] = {(cuuint32_t)kKC, (cuuint32_t)box_rows, (cuuint32_t)kS};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        blast_last_error(__FILE__, __LINE__, "cuTensorMapEncodeTiled failed");
        return BLAST_EDEVICE;
    }
    return BLAST_OK;
}

int bpad_of(int n) { return (n + kM - 1) / kM * kM; }

// Work space of one tensor-core call: coefficient slices, scales, chi weights U.
size_t tc_a_bytes(const blast_plan *p, int Bpad) { return ((size_t)kS * Bpad * p->Kst * 2 + 255) / 256 * 256; }
size_t tc_sa_bytes(int Bpad) { return ((size_t)Bpad * 4 + 255) / 256 * 256; }
// tracers per kind on the tensor-core path (the U and Y tracer dimension)
int tc_mt(const blast_plan *p) { return p->max_clust > p->max_lens ? p->max_clust : p->max_lens; }
int tc_npass(const blast_plan *p) { return p->r_form == 1 ? 4 : 3; }
size_t tc_u_bytes(const blast_plan *p, int Bpad) { return (size_t)Bpad * p->X * 4 * tc_mt(p) * 4; }

template <int KC>
int launch_contract_inst(blast_plan *p, const CUtensorMap &mapB, const CUtensorMap &mapA4, const TcArgs &args,
                         cudaStream_t s)
{
    using C = TcCfg<KC>;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    const int units = args.nbt * args.ngr * args.nqt;
    // persistent CTAs: the autotuned count when set, else every SM
    int grid = p->tune.grid > 0 ? p->tune.grid : sms / args.nbt * args.nbt;
    grid = grid / args.nbt * args.nbt;
    if (grid > units) grid = units;
    if (grid < args.nbt) grid = args.nbt;
    BL_CUDA(allow_opt_in_smem(k_contract_tc<KC>, p->device));
    k_contract_tc<KC><<<grid, kThreads, C::kSmem, s>>>(mapB, mapA4, args);
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}

}  // namespace

// Tensor-core path limits: Chebyshev order <= 96 (coefficient slices and two
// accumulator buffers fit the 512 TMEM columns), n_R a multiple of 32 (whole
// R-tiles), at most 10 tracers of each kind (two groups of five).
bool tc_supported(const blast_plan *p)
{
    return p->Kmma <= 96 && p->Rn % kQT == 0 && p->max_clust <= 2 * kNB && p->max_lens <= 2 * kNB;
}

size_t tc_ws_total(const blast_plan *p, int n)
{
    const int Bpad = bpad_of(n);
    return tc_a_bytes(p, Bpad) + tc_sa_bytes(Bpad) + tc_u_bytes(p, Bpad);
}

int tc_reserve(blast_plan *p, int n) { return p->ws.tc.ensure(tc_ws_total(p, n)); }

// R-tile partials of every pass, then (symmetrised form) the per-order pair
// sums S[b][pass][i][j][es] in FP64
static size_t tc_y_only(const blast_plan *p, int n, int n_esel)
{
    const int ngr = (tc_mt(p) + kNB - 1) / kNB;
    return ((size_t)tc_npass(p) * n_esel * p->X * bpad_of(n) * ngr * (p->Rn / kQT) * kNB * 2 * 4 + 255) / 256 * 256;
}

size_t tc_y_bytes(const blast_plan *p, int n, int n_esel)
{
    const size_t sym = p->r_form == 1 ? (size_t)bpad_of(n) * 4 * tc_mt(p) * tc_mt(p) * n_esel * 8 : 0;
    return tc_y_only(p, n, n_esel) + sym;
}

int launch_basis_slices(blast_plan *p, cudaStream_t s)
{
    k_basis_slices<<<152 * 8, 256, 0, s>>>(p->T64, p->L, p->N, p->Q, p->Kst, p->Tsl, p->scT, p->d_env);
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}

int launch_contract_tc(blast_plan *p, ReqDev *dreq, int n, const int *d_esel, int n_esel, void *ypart,
                       cudaStream_t s)
{
    if (!tc_supported(p)) return BLAST_EINVAL;
    Workspace &ws = p->ws;
    const int Bpad = bpad_of(n);
    int rc;
    if ((rc = ws.tc.ensure(tc_a_bytes(p, Bpad) + tc_sa_bytes(Bpad) + tc_u_bytes(p, Bpad)))) return rc;
    uint16_t *A = ws.tc.as<uint16_t>();
    float *sa = reinterpret_cast<float *>(ws.tc.as<char>() + tc_a_bytes(p, Bpad));
    float *U = reinterpret_cast<float *>(ws.tc.as<char>() + tc_a_bytes(p, Bpad) + tc_sa_bytes(Bpad));
    k_coef_slices<<<Bpad / 8, 256, 0, s>>>(dreq, n, p->N, p->Kst, Bpad, A, sa, p->X, tc_mt(p), U, p->d_env);
    BL_CUDA(cudaGetLastError());

    CUtensorMap mapB;
    if ((rc = make_map(&mapB, p->Tsl, p->Kst, (long long)3 * p->L * p->Q, kQT))) return rc;
    TcArgs args;
    args.reqs = dreq;
    args.n = n;
    args.Bpad = Bpad;
    args.nbt = Bpad / kM;
    args.nqt = p->Q / kQT;
    args.n_esel = n_esel;
    args.L = p->L;
    args.Q = p->Q;
    args.Rn = p->Rn;
    args.RT = p->Rn / kQT;
    args.MT = tc_mt(p);
    args.npass = tc_npass(p);
    args.sym = p->r_form == 1;
    args.X = p->X;
    args.Kst = p->Kst;
    args.Kmma = p->Kmma;
    args.esel = d_esel;
    args.scT = p->scT;
    args.sa = sa;
    args.A = A;
    args.Y = (float *)ypart;
    args.err = p->d_err;
    args.trip = p->test_trip;
    p->test_trip = -1;  // one call only
    args.ngr = (tc_mt(p) + kNB - 1) / kNB;
    if (p->Kst > kKC) {
        // coefficient slice 4 for the shared-memory operand of the p = 4 MMAs
        CUtensorMap mapA4;
        if ((rc = make_map2d(&mapA4, A + (size_t)(kS - 1) * Bpad * p->Kst, p->Kst, Bpad, kM))) return rc;
        return launch_contract_inst<2>(p, mapB, mapA4, args, s);
    }
    return launch_contract_inst<1>(p, mapB, mapB, args, s);
}

int launch_reduce_tc(blast_plan *p, ReqDev *dreq, int n, const int *d_esel, int n_esel, const void *ypart,
                     cudaStream_t s)
{
    const int Bpad = bpad_of(n);
    const float *U =
        reinterpret_cast<const float *>(p->ws.tc.as<char>() + tc_a_bytes(p, Bpad) + tc_sa_bytes(Bpad));
    const int RT = p->Rn / kQT, MT = tc_mt(p), ngr = (MT + kNB - 1) / kNB;
    const int sym = p->r_form == 1, npass = tc_npass(p);
    double *S = sym ? reinterpret_cast<double *>((char *)const_cast<void *>(ypart) + tc_y_only(p, n, n_esel)) : nullptr;
    const size_t stage = ((size_t)RT * kNB * 64 + 2 * MT * 32) * 4 + 8;
    // chi-chunk warps and stages: the autotuned pair when set (and fitting),
    // else 8 warps (4 for large stages) with as many stages as fit two blocks per SM
    int W = stage > 8192 ? 4 : 8;
    int NS = (int)((110 * 1024) / (W * stage));
    if (p->tune.red_w > 0 && p->tune.red_ns > 0 && (size_t)p->tune.red_w * p->tune.red_ns * stage <= 220 * 1024) {
        W = p->tune.red_w;
        NS = p->tune.red_ns;
    }
    if (NS > 4) NS = 4;
    if (NS < 1) return BLAST_EINVAL;
    const size_t smem = (size_t)W * NS * stage;
    dim3 grid((n + 31) / 32, n_esel, npass * ngr);  // cosmology tiles of 32 that hold a request
    if (MT > kNB) {
        BL_CUDA(allow_opt_in_smem(k_reduce_tc<2 * kNB>, p->device));
        k_reduce_tc<2 * kNB><<<grid, 32 * W, smem, s>>>(dreq, (const float *)ypart, U, n, p->X, p->L, d_esel,
                                                       n_esel, RT, MT, Bpad / 32, ngr, NS, p->d_pref, p->d_err, sym,
                                                       S);
    } else {
        BL_CUDA(allow_opt_in_smem(k_reduce_tc<kNB>, p->device));
        k_reduce_tc<kNB><<<grid, 32 * W, smem, s>>>(dreq, (const float *)ypart, U, n, p->X, p->L, d_esel, n_esel,
                                                    RT, MT, Bpad / 32, ngr, NS, p->d_pref, p->d_err, sym, S);
    }
    BL_CUDA(cudaGetLastError());
    if (sym) {
        const int pmax = blast_npairs(p->max_clust, p->max_lens);
        k_sym_combine<<<dim3((pmax * n_esel + 127) / 128, n), 128, 0, s>>>(dreq, S, MT, d_esel, n_esel);
        BL_CUDA(cudaGetLastError());
    }
    return BLAST_OK;
}
