// Tensor-core contraction (a) with the R-sum of quadrature (b) fused into the
// epilogue, for a batch of cosmologies:
//
//   w_b(t, l, q) = sum_n a_b[n] T~[t][l][n][q]                       (Eq. pmd)
//   Y_b(t, l, a, rt, j) = sum_{r in R-tile rt} V_bj(a, r) w_b(t, l, a n_R + r)
//
// as one GEMM per (t, l): M = cosmologies (128 per CTA, TMEM lanes), N = 32
// chi-R nodes (one R-tile), K = Chebyshev order.  The expansion of P in
// Chebyshev polynomials cancels strongly where P is small (high l, low-z
// lensing), so an FP32-accumulated hi/lo split is not accurate enough.
// Instead both operands are cut into S = 5 fixed-point slices of 8 bits:
//
//   a_b[n]     = 2^ea(b)    sum_p 2^(-8(p+1)) A_p[b][n],   A_p integers, |A_p| <= 256
//   T~[.][n][q] = 2^eT(col) sum_p 2^(-8(p+1)) T_p[col][n]
//
// Slice p is stored as A_p 2^(-8p) (T_q 2^(-8q)): an integer of at most 9
// bits times a power of two, exact in BF16.  Every product is exact, and level
// k, D_k 2^(-8k) = sum_{p+q=k} sum_n (A_p 2^-8p)(T_q 2^-8q), is a multiple of
// 2^(-8k) below 2^(23-8k) in magnitude, so the FP32 tensor-core accumulation
// is exact.  The 15 slice pairs p+q <= 4 feed 5 level accumulators in TMEM;
// the epilogue adds the levels with a cascade of fast two-sums, each exact for
// operands on these grids, W 2^-32 = m + (e1 + e2 + e3 + e4), and scales by
// 2^(ea + eT - 16).  The R sum that follows also cancels (w oscillates around
// R = 1), so it runs on unevaluated pairs: exact products (FMA), two products
// (columns two R nodes apart) added plainly, and two-sum accumulation of those
// sums, two columns at a time in packed FP32 pairs; the pairs reach the chi
// sum intact.
//
// Warp roles (576 threads): warp 0 issues TMA loads of the basis slices,
// warp 1 owns TMEM and issues tcgen05.mma (A = coefficient slices resident in
// TMEM, B = basis slices in shared memory), warps 2..17 run the epilogue (one
// TMEM lane = one cosmology per thread, four warps per lane quadrant, joined
// by a named barrier per quadrant).  Every mbarrier wait is bounded; on
// timeout the kernel records an error code in host-mapped memory and exits.
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
constexpr int kKC = 64;                   // K elements per 128-byte swizzle row
constexpr int kStages = 4;
constexpr int kEP = 4;                    // epilogue warps per TMEM lane quadrant
constexpr int kThreads = 64 + 128 * kEP;  // 2 control warps + 16 epilogue warps
constexpr int kHC = 32 / kEP;             // columns per epilogue thread
constexpr int kNB = 5;                    // B-side tracers handled per thread (registers)
constexpr uint32_t kACol = 2 * kS * kQT;          // TMEM column of the coefficient slices
constexpr uint32_t kBSliceBytes = kQT * 128;      // 32 rows x 64 bf16
constexpr uint32_t kBStageBytes = kS * kBSliceBytes;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kCtrlBytes = 256;               // mbarriers, TMEM address, abort flag
constexpr long long kWaitLimit = 4000000000LL;  // clock cycles (about 2 s)
constexpr uint32_t kSuspendNs = 1000000;        // longest suspension of one phase test

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
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned sleep_ns = 0)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitLimit) return false;
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

// True in exactly one lane of the (converged) warp.
__device__ __forceinline__ bool elect_one()
{
    uint32_t p;
    asm volatile("{\n\t.reg .pred P;\n\telect.sync _|P, 0xffffffff;\n\tselp.u32 %0, 1, 0, P;\n\t}\n" : "=r"(p));
    return p != 0;
}

// Thirty-two consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]),
        "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// Four consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
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

// Wait for this thread's TMEM loads of four columns per level; the registers
// they fill are operands, so no use of them can move above the wait.
__device__ __forceinline__ void tmem_wait_ld4(uint32_t (&r)[BLAST_TC_SLICES][4])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0][0]), "+r"(r[0][1]), "+r"(r[0][2]), "+r"(r[0][3]), "+r"(r[1][0]), "+r"(r[1][1]),
                   "+r"(r[1][2]), "+r"(r[1][3]), "+r"(r[2][0]), "+r"(r[2][1]), "+r"(r[2][2]), "+r"(r[2][3]),
                   "+r"(r[3][0]), "+r"(r[3][1]), "+r"(r[3][2]), "+r"(r[3][3]), "+r"(r[4][0]), "+r"(r[4][1]),
                   "+r"(r[4][2]), "+r"(r[4][3])
                 :
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

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

// Coefficient slices, one warp per cosmology: A_p[b][n] and 2^ea(b); also the
// chi weights U transposed to cosmology-fastest order for the reduction.
__global__ void k_coef_slices(const ReqDev *__restrict__ reqs, int n, int N, int Kp, int Bpad, uint16_t *A,
                              float *sa, int X, int ntr_max, float *UT, float *UTl)
{
    const int b = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (b >= Bpad) return;
    const double *a = (b < n) ? reqs[b].a64 : nullptr;
    double mx = 0.0;
    for (int k = lane; k < N; k += 32) mx = fmax(mx, fabs(a ? a[k] : 0.0));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
    for (int k = lane; k < Kp; k += 32) {
        uint16_t s[kS];
        slice8((a && k < N) ? ldexp(a[k], -e) : 0.0, s);
#pragma unroll
        for (int p = 0; p < kS; p++) A[((size_t)p * Bpad + b) * Kp + k] = s[p];
    }
    if (lane == 0) sa[b] = ldexpf(1.0f, e);
    const int ntr = (b < n) ? reqs[b].n_clust + reqs[b].n_lens : 0;
    const double *U = (b < n) ? reqs[b].U64 : nullptr;
    for (int i = lane; i < ntr_max * X; i += 32) {
        const double u = (i < ntr * X) ? U[i] : 0.0;
        const float uh = (float)u;
        UT[(size_t)i * Bpad + b] = uh;
        UTl[(size_t)i * Bpad + b] = (float)(u - (double)uh);
    }
}

// Basis slices, one warp per tile of kQT columns (t, l, q0..q0+31), a lane per
// column: T_p[col][n] 2^(-8p) 2^(eT(col) - eG) with eG the largest column
// exponent of the tile, and one scale 2^(eG - 16) per tile.  A column keeps
// its own 40-bit fixed-point precision; the power of two moves the exponent
// only.  Columns more than 2^90 below the tile's largest (or in tiles whose
// scale underflows FP32) are zero: they could not change the tile's sum.
__global__ void k_basis_slices(const double *__restrict__ T, int L, int N, int Q, int Kp, uint16_t *Tsl, float *scT)
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
        for (int k = 0; k < N; k++) mx = fmax(mx, fabs(src[(size_t)k * Q]));
        int e = 0;
        if (mx > 0.0) frexp(mx, &e);
        int eG = (mx > 0.0) ? e : INT_MIN;
        for (int o = 16; o; o >>= 1) eG = max(eG, __shfl_xor_sync(0xffffffffu, eG, o));
        const float scf = (eG != INT_MIN) ? (float)ldexp(1.0, eG - 16) : 0.0f;
        const bool keep = mx > 0.0 && scf != 0.0f && e - eG >= -90;
        const float shift = keep ? ldexpf(1.0f, e - eG) : 0.0f;
        for (int k = 0; k < Kp; k++) {
            uint16_t s[kS];
            slice8((k < N && keep) ? ldexp(src[(size_t)k * Q], -e) : 0.0, s, shift);
#pragma unroll
            for (int p = 0; p < kS; p++) Tsl[((size_t)p * ncol + col) * Kp + k] = s[p];
        }
        if (lane == 0) scT[tile] = scf;
    }
}

// ---------------------------------------------------------------- main kernel
struct TcArgs {
    const ReqDev *reqs;
    int n, Bpad, nbt, nqt, n_esel, L, Q, Rn, RT, MT;
    const int *esel;
    const float *scT;    // [3][L][Q / kQT] one scale per tile
    const float *sa;     // [Bpad]
    const uint16_t *A;   // [S][Bpad][64] coefficient slices
    float *Y;            // [3][n_esel][X][n][RT][MT] pairs (hi, lo)
    int *err;            // host-mapped error word
};

__global__ void __launch_bounds__(kThreads, 1)
k_contract_tc(const __grid_constant__ CUtensorMap mapB, TcArgs args)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment for the swizzled tiles
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sB = smem;                                  // kStages x kS x 4 KB
    uint64_t *bars = (uint64_t *)(sB + kStages * kBStageBytes);  // kCtrlBytes of control words
    uint64_t *full = bars, *empty = bars + kStages, *aready = bars + 2 * kStages;
    uint64_t *tfull = aready + 1, *tempty = tfull + 2;
    uint32_t *tmem_slot = (uint32_t *)(tempty + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    float *ybuf = (float *)((unsigned char *)bars + kCtrlBytes);   // [2][kEP-1][2 kNB][kM] partial pairs
    f32x2 *vsm = (f32x2 *)(ybuf + 2 * (kEP - 1) * 2 * kNB * kM);   // [kNB][kHC/2][128 kEP] weights

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int btile = blockIdx.x % args.nbt;
    const int n_iter_unit = 3 * args.n_esel;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; i++) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        mbar_init(aready, 128);
        for (int i = 0; i < 2; i++) {
            mbar_init(&tfull[i], 1); mbar_init(&tempty[i], 128 * kEP);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
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
        uint32_t g = 0;
        bool ok = true;
        for (int u = blockIdx.x; ok && u < args.nbt * args.nqt; u += gridDim.x) {
            const int q0 = (u / args.nbt) * kQT;
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
                    const int t = it / args.n_esel, e = args.esel[it % args.n_esel];
                    const int row = (t * args.L + e) * args.Q + q0;
                    mbar_expect_tx(&full[st], kBStageBytes);
                    tma_load_3d(sB + st * kBStageBytes, &mapB, &full[st], 0, row, 0);
                }
                __syncwarp();
            }
        }
        // drain: every issued load has landed before the CTA may exit
        for (uint32_t h = (g > kStages ? g - kStages : 0); h < g; h++)
            mbar_wait(&full[h % kStages], (h / kStages) & 1, 64);
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (whole warp waits; each MMA is
        // issued by one elected lane of the converged warp)
        bool ok = __all_sync(0xffffffffu, mbar_wait(aready, 0, 64));  // coefficient slices in TMEM
        if (!ok && lane == 0) { atomicExch(args.err, 2); *abort_flag = 1; }
        tc_fence_after();
        const uint32_t b0 = __shfl_sync(0xffffffffu, smem_u32(sB), 0);  // warp-uniform operands
        const uint32_t tm = __shfl_sync(0xffffffffu, tmem, 0);
        uint32_t g = 0;
        for (int u = blockIdx.x; ok && u < args.nbt * args.nqt; u += gridDim.x) {
            for (int it = 0; it < n_iter_unit; it++, g++) {
                const int st = g % kStages;
                const uint32_t ph = (g / kStages) & 1;
                const int buf = g & 1;
                const uint32_t tph = (g >> 1) & 1;
                const bool bad = *abort_flag || !mbar_wait(&full[st], ph, 64) || !mbar_wait(&tempty[buf], tph ^ 1, 64);
                if (__any_sync(0xffffffffu, bad)) {
                    if (lane == 0) { atomicExch(args.err, 3); *abort_flag = 1; }
                    ok = false;
                    break;
                }
                tc_fence_after();
                // operands of the 60 MMAs: accumulator levels of this buffer, coefficient
                // slices in TMEM, basis slice descriptors offset from this stage's first
                const uint32_t dbase = tm + buf * (kS * kQT);
                const uint64_t bbase = sdesc(b0 + st * kBStageBytes);
                if (elect_one()) {
#pragma unroll
                    for (int lev = 0; lev < kS; lev++) {
#pragma unroll
                        for (int p = 0; p <= lev; p++) {
                            const int q = lev - p;
#pragma unroll
                            for (int kk = 0; kk < kKC / 16; kk++)
                                umma_ts(dbase + lev * kQT, tm + kACol + p * (kKC / 2) + kk * 8,
                                        bbase + (uint64_t)((q * kBSliceBytes + kk * 32) >> 4), (p > 0 || kk > 0) ? 1u : 0u);
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
    } else {
        // ------------------------------------------------ epilogue: kEP warps per TMEM lane quadrant;
        // a thread owns one cosmology (TMEM lane) and kHC of the tile's 32 columns.
        const int ew = warp - 2;
        const int quad = warp & 3;   // lanes 32 quad .. 32 quad + 31 are readable by this warp
        const int part = ew >> 2;    // columns [kHC part, kHC part + kHC)
        const int bl_ = quad * 32 + lane;
        const int b = btile * kM + bl_;
        const bool valid = b < args.n;
        const ReqDev *rq = valid ? &args.reqs[b] : nullptr;
        const int ng = valid ? rq->n_clust : 0, ns = valid ? rq->n_lens : 0;
        const float sa = args.sa[b];
        const uint32_t lane_addr = ((uint32_t)(quad * 32)) << 16;
        const int cb = part * kHC;
        if (part == 0) {
            // coefficient slices of cosmology b -> TMEM lane b, columns kACol + 32 p ..
#pragma unroll 1
            for (int p = 0; p < kS; p++) {
                uint32_t r[32];
                const uint4 *src = reinterpret_cast<const uint4 *>(args.A + ((size_t)p * args.Bpad + b) * kKC);
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const uint4 v = __ldg(src + i);
                    r[4 * i] = v.x; r[4 * i + 1] = v.y; r[4 * i + 2] = v.z; r[4 * i + 3] = v.w;
                }
                tmem_st32(tmem + lane_addr + kACol + p * (kKC / 2), r);
            }
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(aready);
        }
        // Every thread of the quadrant's four warps passes the same number of
        // named barriers; after a wait runs out the warps skip the work but keep
        // the count, so no barrier is left waiting.
        const int bar_id = 1 + quad;
        uint32_t g = 0;
        bool dead = false;
        for (int u = blockIdx.x; u < args.nbt * args.nqt; u += gridDim.x) {
            const int q0 = (u / args.nbt) * kQT;
            const int a = q0 / args.Rn, rt = (q0 % args.Rn) / kQT;
            // quadrature weights of this cosmology times its scale 2^ea, kept in this
            // thread's own slots of shared memory (read back only by this thread)
            f32x2 *vme = vsm + (threadIdx.x - 64);
            for (int t = 0; t < 3; t++) {
                const int offB = (t == 0) ? 0 : ng, nB = (t == 0) ? ng : ns;
                if (t < 2) {
#pragma unroll
                    for (int j = 0; j < kNB; j++) {
                        const float4 *src =
                            (valid && j < nB)
                                ? reinterpret_cast<const float4 *>(rq->V32 + (size_t)(offB + j) * args.Q + q0 + cb)
                                : nullptr;
#pragma unroll
                        for (int c = 0; c < kHC / 4; c++) {
                            const float4 v = src ? src[c] : make_float4(0.f, 0.f, 0.f, 0.f);
                            vme[(j * (kHC / 2) + 2 * c) * (128 * kEP)] = pk2(v.x * sa, v.y * sa);
                            vme[(j * (kHC / 2) + 2 * c + 1) * (128 * kEP)] = pk2(v.z * sa, v.w * sa);
                        }
                    }
                }
                for (int es = 0; es < args.n_esel; es++, g++) {
                    const int buf = g & 1;
                    const uint32_t tph = (g >> 1) & 1;
                    if (!dead) {
                        bool lost = *abort_flag != 0;
                        if (!lost && !mbar_wait(&tfull[buf], tph)) {
                            lost = true;
                            atomicExch(args.err, 4);
                            *abort_flag = 1;
                        }
                        dead = __any_sync(0xffffffffu, lost);
                    }
                    float Sh[kNB], Sl[kNB];
#pragma unroll
                    for (int j = 0; j < kNB; j++) { Sh[j] = 0.f; Sl[j] = 0.f; }
                    if (!dead) {
                        tc_fence_after();
                        const uint32_t tcol = tmem + lane_addr + buf * (kS * kQT) + cb;
                        // R-sum of this thread's columns, two columns per packed lane pair, as
                        // negated unevaluated sums An + Bn: each product V w is split exactly
                        // (FMA) and each addition's rounding error is kept (two-sum), so the
                        // sum survives the cancellation of oscillating w
                        f32x2 An[kNB], Bn[kNB];
                        // four columns (two packed pairs) per step: pair A = columns c0, c0+1
                        // in lanes x, y; pair B = c0+2, c0+3.  Each lane's two exact products
                        // (columns two R nodes apart) are added plainly, and that sum enters
                        // the compensated sum
#pragma unroll
                        for (int c0 = 0; c0 < kHC; c0 += 4) {
                            uint32_t D[kS][4];
#pragma unroll
                            for (int lev = 0; lev < kS; lev++) tmem_ld4(tcol + lev * kQT + c0, D[lev]);
                            tmem_wait_ld4(D);
                            if (c0 + 4 == kHC) {  // every level of this buffer is in registers: release it
                                tc_fence_before();
                                mbar_arrive(&tempty[buf]);
                            }
                            // Level k holds D_k 2^(-8k) 2^(eT - eG), an integer multiple of
                            // 2^(-8k) 2^(eT - eG) below 2^(23-8k) 2^(eT - eG) in magnitude, so
                            // every fast two-sum of the cascade is exact:
                            // W 2^(eT - eG - 32) = m + (e1 + e2 + e3 + e4), one rounding in the
                            // low part only
                            f32x2 m[2], lo[2];
#pragma unroll
                            for (int h = 0; h < 2; h++) {
                                f32x2 d[kS];
#pragma unroll
                                for (int lev = 0; lev < kS; lev++)
                                    d[lev] = pk2(__uint_as_float(D[lev][2 * h]), __uint_as_float(D[lev][2 * h + 1]));
                                f32x2 e1, e2, e3, e4;
                                fast_two_sum2(d[0], d[1], m[h], e1);
                                fast_two_sum2(m[h], d[2], m[h], e2);
                                fast_two_sum2(m[h], d[3], m[h], e3);
                                fast_two_sum2(m[h], d[4], m[h], e4);
                                lo[h] = add2(add2(e1, e2), add2(e3, e4));
                            }
                            const f32x2 mn0 = neg2(m[0]), mn1 = neg2(m[1]);
#pragma unroll
                            for (int j = 0; j < kNB; j++) {
                                const f32x2 v0 = vme[(j * (kHC / 2) + c0 / 2) * (128 * kEP)];
                                const f32x2 v1 = vme[(j * (kHC / 2) + c0 / 2 + 1) * (128 * kEP)];
                                const f32x2 p0 = mul2(v0, mn0), p1 = mul2(v1, mn1);  // -fl(v m)
                                const f32x2 e0 = fma2(v0, lo[0], fma2(v0, m[0], p0));  // v lo + (v m - fl(v m))
                                const f32x2 e1 = fma2(v1, lo[1], fma2(v1, m[1], p1));
                                const f32x2 ps = add2(p0, p1), pe = add2(e0, e1);
                                if (c0 == 0) {  // the sums start here
                                    An[j] = ps;
                                    Bn[j] = neg2(pe);
                                } else {
                                    f32x2 se;
                                    two_sum2(An[j], ps, An[j], se);
                                    Bn[j] = add2(Bn[j], sub2(se, pe));
                                }
                            }
                        }
                        // both lanes into one pair per tracer: S = -(An.x + An.y) - (Bn.x + Bn.y)
#pragma unroll
                        for (int j = 0; j < kNB; j++) {
                            const float2 A2 = unpk2(An[j]), B2 = unpk2(Bn[j]);
                            float h, el;
                            two_sum(A2.x, A2.y, h, el);
                            Sh[j] = -h;
                            Sl[j] = -__fadd_rn(el, __fadd_rn(B2.x, B2.y));
                        }
                    }
                    // add the column parts: parts 1.. hand their pairs to part 0 through
                    // shared memory ([part - 1][2 kNB][kM], double buffered by iteration)
                    float *yq = ybuf + (size_t)(g & 1) * (kEP - 1) * 2 * kNB * kM;
                    if (part > 0) {
                        float *slot = yq + (size_t)(part - 1) * 2 * kNB * kM + bl_;
#pragma unroll
                        for (int j = 0; j < kNB; j++) { slot[j * kM] = Sh[j]; slot[(kNB + j) * kM] = Sl[j]; }
                    }
                    named_bar_sync(bar_id, 32 * kEP);
                    if (part == 0 && !dead) {
#pragma unroll
                        for (int q = 0; q < kEP - 1; q++) {
                            const float *slot = yq + (size_t)q * 2 * kNB * kM + bl_;
#pragma unroll
                            for (int j = 0; j < kNB; j++) {
                                float se;
                                two_sum(Sh[j], slot[j * kM], Sh[j], se);
                                Sl[j] = __fadd_rn(Sl[j], __fadd_rn(se, slot[(kNB + j) * kM]));
                            }
                        }
                        if (valid) {
                            // the tile's scale 2^(eG - 16) (exact), then the pair (hi, lo)
                            // of tracer j at j and MT + j
                            const float tsc =
                                args.scT[((size_t)t * args.L + args.esel[es]) * (args.Q / kQT) + q0 / kQT];
#pragma unroll
                            for (int j = 0; j < kNB; j++) { Sh[j] *= tsc; Sl[j] *= tsc; }
                            // Y[t][es][a][b][rt][j] pairs (hi, lo): one cosmology's R tiles of a
                            // chi node are contiguous for the reduction's vector loads
                            float2 *y = reinterpret_cast<float2 *>(args.Y) +
                                        ((((size_t)t * args.n_esel + es) * (args.Q / args.Rn) + a) * args.n + b) *
                                            (size_t)(args.RT * args.MT) + (size_t)rt * args.MT;
#pragma unroll
                            for (int j = 0; j < kNB; j++)
                                if (j < args.MT) y[j] = make_float2(Sh[j], Sl[j]);
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

// A thread's staging slot of k_reduce_tc in float2 units: RT MT pairs and the
// kNB + kNB chi weights, rounded up to 16 bytes so every slot is 16-byte aligned.
__host__ __device__ __forceinline__ int reduce_slot_f2(int RT, int MT) { return (RT * MT + kNB + 1) & ~1; }

// Asynchronous global -> shared copies (cp.async): 16, 8 or 4 bytes each,
// visible to the issuing thread after the matching wait_group.
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Sum over R tiles and chi nodes for the tensor-core path, one thread per
// (cosmology, type, ell, chi chunk) accumulating every tracer pair (i, j):
//   s_j(a) = sum_rt Y(t, l, a, rt, j)          (pairs (hi, lo), two-sum)
//   C_ij(l) = N_AB(l) sum_a U_i(a) s_j(a)      (exact products, two-sum)
// A block is 32 cosmologies x W chi chunks (one warp each).  Each thread
// streams its own R-tile pairs and chi weights of the next STG - 1 chi nodes
// into its own shared-memory slots with cp.async while it sums the current
// one, so enough bytes are in flight to keep HBM busy; the chunks are then
// added in a tree through the same shared memory.
template <int W, int STG>
__global__ void __launch_bounds__(32 * W, 2)
k_reduce_tc(const ReqDev *__restrict__ reqs, const float *__restrict__ Y, const float *__restrict__ UT,
            const float *__restrict__ UTl, int n, int Bpad, int X, int L, const int *__restrict__ esel, int n_esel,
            int RT, int MT, const double *__restrict__ pref)
{
    extern __shared__ __align__(16) unsigned char red_smem[];
    const int lane = threadIdx.x & 31, chunk = threadIdx.x >> 5;
    const int b = blockIdx.x * 32 + lane;
    const int es = blockIdx.y, t = blockIdx.z;
    const ReqDev *rq = (b < n) ? &reqs[b] : nullptr;
    const int ng = rq ? rq->n_clust : 0, ns = rq ? rq->n_lens : 0;
    const int nA = (t == 2) ? ns : ng, nB = (t == 0) ? ng : ns, offA = (t == 2) ? ng : 0;
    const int e = esel[es];
    const int col = rq ? rq->e_out[e] : -1;
    const bool active = rq && nA > 0 && nB > 0 && col >= 0;
    // per thread and stage: RT MT pairs (hi, lo), then U hi[kNB], U lo[kNB]
    const int RTMT = RT * MT;
    const int slot_f2 = reduce_slot_f2(RT, MT);
    float2 *my = reinterpret_cast<float2 *>(red_smem) + ((size_t)chunk * STG * 32 + lane) * slot_f2;
    auto stage_ptr = [&](int st) { return my + (size_t)st * 32 * slot_f2; };
    const int per = (X + W - 1) / W;
    const int a0 = chunk * per, a1 = min(X, a0 + per);
    const int cnt = active ? max(0, a1 - a0) : 0;
    const float2 *Yb = reinterpret_cast<const float2 *>(Y) + ((size_t)t * n_esel + es) * (size_t)X * n * RTMT +
                       (size_t)b * RTMT;
    const bool even = (RTMT & 1) == 0;  // 16-byte copies when each thread's pairs are 16-byte aligned
    auto issue = [&](int k) {           // copies of chi node a0 + k into stage k % STG
        if (k < cnt) {
            float2 *d = stage_ptr(k % STG);
            const float2 *y = Yb + (size_t)(a0 + k) * n * RTMT;
            if (even)
                for (int i = 0; i < RTMT; i += 2) cp_async16(d + i, y + i);
            else
                for (int i = 0; i < RTMT; i++) cp_async8(d + i, y + i);
            float *u = reinterpret_cast<float *>(d + RTMT);
            for (int i = 0; i < nA; i++) {
                const size_t ui = ((size_t)(offA + i) * X + a0 + k) * Bpad + b;
                cp_async4(u + i, UT + ui);
                cp_async4(u + kNB + i, UTl + ui);
            }
        }
        cp_async_commit();  // every thread commits every step: group counts stay uniform
    };
    float Zh[kNB][kNB], Zl[kNB][kNB];
#pragma unroll
    for (int i = 0; i < kNB; i++)
#pragma unroll
        for (int j = 0; j < kNB; j++) { Zh[i][j] = 0.f; Zl[i][j] = 0.f; }
#pragma unroll
    for (int k = 0; k < STG - 1; k++) issue(k);
    for (int k = 0; k < per; k++) {
        issue(k + STG - 1);
        cp_async_wait<STG - 1>();  // node a0 + k has landed
        if (k >= cnt) continue;
        const float2 *v = stage_ptr(k % STG);
        float sh[kNB], sl[kNB];
#pragma unroll
        for (int j = 0; j < kNB; j++) { sh[j] = 0.f; sl[j] = 0.f; }
        for (int rt = 0; rt < RT; rt++) {
#pragma unroll
            for (int j = 0; j < kNB; j++) {
                if (j < nB) {
                    const float2 y = v[rt * MT + j];
                    float se;
                    two_sum(sh[j], y.x, sh[j], se);
                    sl[j] = __fadd_rn(sl[j], __fadd_rn(se, y.y));
                }
            }
        }
        const float *u = reinterpret_cast<const float *>(v + RTMT);
        float sv[kNB], sle[kNB];
#pragma unroll
        for (int j = 0; j < kNB; j++) two_sum(sh[j], sl[j], sv[j], sle[j]);
#pragma unroll
        for (int i = 0; i < kNB; i++) {
            if (i >= nA) continue;
            const float uh = u[i], ul = u[kNB + i];
#pragma unroll
            for (int j = 0; j < kNB; j++) {
                if (j >= nB) continue;
                const float pr = __fmul_rn(uh, sv[j]);
                const float pe = fmaf(uh, sle[j], fmaf(ul, sv[j], fmaf(uh, sv[j], -pr)));
                float se;
                two_sum(Zh[i][j], pr, Zh[i][j], se);
                Zl[i][j] = __fadd_rn(Zl[i][j], __fadd_rn(se, pe));
            }
        }
    }
    cp_async_wait<0>();
    __syncthreads();  // the staging slots become the tree's exchange area
    // tree over the chi chunks: the upper half of the warps hands its pairs down
    float(*red)[32][2 * kNB * kNB] = reinterpret_cast<float(*)[32][2 * kNB * kNB]>(red_smem);
    for (int half = W / 2; half >= 1; half >>= 1) {
        if (chunk >= half && chunk < 2 * half) {
#pragma unroll
            for (int i = 0; i < kNB; i++)
#pragma unroll
                for (int j = 0; j < kNB; j++) {
                    red[chunk - half][lane][2 * (i * kNB + j)] = Zh[i][j];
                    red[chunk - half][lane][2 * (i * kNB + j) + 1] = Zl[i][j];
                }
        }
        __syncthreads();
        if (chunk < half) {
#pragma unroll
            for (int i = 0; i < kNB; i++)
#pragma unroll
                for (int j = 0; j < kNB; j++) {
                    float se;
                    two_sum(Zh[i][j], red[chunk][lane][2 * (i * kNB + j)], Zh[i][j], se);
                    Zl[i][j] = __fadd_rn(Zl[i][j], __fadd_rn(se, red[chunk][lane][2 * (i * kNB + j) + 1]));
                }
        }
        __syncthreads();
    }
    if (chunk != 0 || !active) return;
    const double pf = pref[t * L + e];
    const int ngg = ng * (ng + 1) / 2, ngs = ng * ns;
#pragma unroll
    for (int i = 0; i < kNB; i++) {
#pragma unroll
        for (int j = 0; j < kNB; j++) {
            if (i >= nA || j >= nB) continue;
            int p;
            if (t == 0) { if (i > j) continue; p = i * ng - i * (i - 1) / 2 + (j - i); }
            else if (t == 1) p = ngg + i * ns + j;
            else { if (i > j) continue; p = ngg + ngs + i * ns - i * (i - 1) / 2 + (j - i); }
            double out = pf * ((double)Zh[i][j] + (double)Zl[i][j]);
            if (rq->status) out = nan("");
            rq->cl[(size_t)p * rq->n_sel + col] = out;
        }
    }
}

// Shared memory of k_reduce_tc<W, STG>: the staging slots, at least the tree's area.
size_t reduce_smem(int W, int STG, int RT, int MT)
{
    const size_t stage = (size_t)W * STG * 32 * reduce_slot_f2(RT, MT) * sizeof(float2);
    const size_t tree = (size_t)(W / 2) * 32 * 2 * kNB * kNB * sizeof(float);
    return stage > tree ? stage : tree;
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 3-D map over [S][rows][Kp] bf16, box {64, box_rows, S}, 128-byte swizzle.
int make_map(CUtensorMap *m, void *base, int Kp, long long rows, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return BLAST_EDEVICE;
    cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)kS};
    cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
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

// Work space of one tensor-core call: coefficient slices, scales, transposed U.
size_t tc_ws_bytes(const blast_plan *p, int Bpad)
{
    return (size_t)kS * Bpad * p->Kp * 2 + (size_t)Bpad * 4 +
           2 * (size_t)(p->max_clust + p->max_lens) * p->X * Bpad * 4 + 256;
}

size_t tc_smem_bytes()
{
    return 1024 + kStages * kBStageBytes + kCtrlBytes + 2 * (kEP - 1) * 2 * kNB * kM * sizeof(float) +
           kNB * (kHC / 2) * 128 * kEP * sizeof(f32x2);
}

}  // namespace

bool tc_supported(const blast_plan *p)
{
    return p->Kp == kKC && p->Rn % kQT == 0 && p->max_clust <= kNB && p->max_lens <= kNB;
}

int launch_basis_slices(blast_plan *p, cudaStream_t s)
{
    k_basis_slices<<<152 * 8, 256, 0, s>>>(p->T64, p->L, p->N, p->Q, p->Kp, p->Tsl, p->scT);
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}

int launch_contract_tc(blast_plan *p, ReqDev *dreq, int n, const int *d_esel, int n_esel, void *ypart,
                       cudaStream_t s)
{
    if (!tc_supported(p)) return BLAST_EINVAL;
    Workspace &ws = p->ws;
    const int Bpad = (n + kM - 1) / kM * kM;
    int rc;
    const int ntr_max = p->max_clust + p->max_lens;
    if ((rc = ws.tc.ensure(tc_ws_bytes(p, Bpad)))) return rc;
    uint16_t *A = ws.tc.as<uint16_t>();
    float *sa = reinterpret_cast<float *>(A + (size_t)kS * Bpad * p->Kp);
    float *UT = sa + Bpad;
    float *UTl = UT + (size_t)ntr_max * p->X * Bpad;
    k_coef_slices<<<Bpad / 8, 256, 0, s>>>(dreq, n, p->N, p->Kp, Bpad, A, sa, p->X, ntr_max, UT, UTl);
    BL_CUDA(cudaGetLastError());

    CUtensorMap mapB;
    if ((rc = make_map(&mapB, p->Tsl, p->Kp, (long long)3 * p->L * p->Q, kQT))) return rc;
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
    args.MT = p->max_tr;
    args.esel = d_esel;
    args.scT = p->scT;
    args.sa = sa;
    args.A = A;
    args.Y = (float *)ypart;
    args.err = p->d_err;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    int units = args.nbt * args.nqt;
    int grid = sms / args.nbt * args.nbt;
    if (grid > units) grid = units;
    if (grid < args.nbt) grid = args.nbt;
    size_t smem = tc_smem_bytes();
    BL_CUDA(cudaFuncSetAttribute(k_contract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_contract_tc<<<grid, kThreads, smem, s>>>(mapB, args);
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}

int launch_reduce_tc(blast_plan *p, ReqDev *dreq, int n, const int *d_esel, int n_esel, const void *ypart,
                     cudaStream_t s)
{
    const int Bpad = (n + kM - 1) / kM * kM;
    const float *UT = reinterpret_cast<const float *>(p->ws.tc.as<uint16_t>() + (size_t)kS * Bpad * p->Kp) + Bpad;
    const float *UTl = UT + (size_t)(p->max_clust + p->max_lens) * p->X * Bpad;
    const int RT = p->Rn / kQT, MT = p->max_tr;
    dim3 grid((n + 31) / 32, n_esel, 3);
    constexpr size_t kSmemMax = 220 * 1024;
    if (reduce_smem(8, 2, RT, MT) <= kSmemMax / 2) {  // 8 chi chunks, 2 stages, two blocks per SM
        const int smem = (int)reduce_smem(8, 2, RT, MT);
        BL_CUDA(cudaFuncSetAttribute(k_reduce_tc<8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        k_reduce_tc<8, 2><<<grid, 32 * 8, smem, s>>>(dreq, (const float *)ypart, UT, UTl, n, Bpad, p->X, p->L, d_esel,
                                                     n_esel, RT, MT, p->d_pref);
    } else {  // long R-tile rows (n_R up to 512): 4 chunks, 2 stages
        const int smem = (int)reduce_smem(4, 2, RT, MT);
        if ((size_t)smem > kSmemMax) return BLAST_EINVAL;
        BL_CUDA(cudaFuncSetAttribute(k_reduce_tc<4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        k_reduce_tc<4, 2><<<grid, 32 * 4, smem, s>>>(dreq, (const float *)ypart, UT, UTl, n, Bpad, p->X, p->L, d_esel,
                                                     n_esel, RT, MT, p->d_pref);
    }
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}
