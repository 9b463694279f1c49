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
// Every slice value is an integer held exactly in BF16, every product is
// exact, and each level D_k = sum_{p+q=k} sum_n A_p T_q stays below 2^24, so
// the FP32 tensor-core accumulation is exact.  The 15 slice pairs p+q <= 4
// feed 5 level accumulators in TMEM; the epilogue combines the levels exactly
// in 64-bit integers, W = sum_k D_k 2^(8(4-k)), rounds once to FP32 and scales
// by 2^(ea + eT - 48).
//
// Warp roles (192 threads): warp 0 issues TMA loads of the basis slices,
// warp 1 owns TMEM and issues tcgen05.mma, warps 2..5 run the epilogue (one
// TMEM lane = one cosmology per thread).  Every mbarrier wait is bounded; on
// timeout the kernel records an error code in host-mapped memory and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "blast_internal.h"

namespace {

constexpr int kS = BLAST_TC_SLICES;       // slices per operand
constexpr int kQT = 32;                   // chi-R nodes per tile (MMA N)
constexpr int kM = 128;                   // cosmologies per tile (MMA M)
constexpr int kKC = 64;                   // K elements per 128-byte swizzle row
constexpr int kStages = 4;
constexpr int kThreads = 192;
constexpr int kMaxTr = BLAST_MAX_TRACERS / 2;
constexpr int kNB = 5;                    // B-side tracers handled per thread (registers)
constexpr uint32_t kASliceBytes = kM * 128;       // 128 rows x 64 bf16
constexpr uint32_t kBSliceBytes = kQT * 128;      // 32 rows x 64 bf16
constexpr uint32_t kBStageBytes = kS * kBSliceBytes;
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitLimit = 4000000000LL;  // clock cycles (about 2 s)

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

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on a phase: false if it did not complete within kWaitLimit cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitLimit) return false;
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

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d_tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
}

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

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---------------------------------------------------------------- slicing
// x (|x| < 2^e) -> S integers in [-256, 256], each exact in BF16.
__device__ __forceinline__ void slice8(double xn, uint16_t (&out)[kS])
{
    double r = xn * 256.0;
#pragma unroll
    for (int p = 0; p < kS; p++) {
        double q = rint(r);
        out[p] = __bfloat16_as_ushort(__float2bfloat16_rn((float)q));
        r = (r - q) * 256.0;
    }
}

// Coefficient slices, one warp per cosmology: A_p[b][n] and 2^ea(b).
__global__ void k_coef_slices(const ReqDev *__restrict__ reqs, int n, int N, int Kp, int Bpad, uint16_t *A,
                              float *sa)
{
    const int b = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (b >= Bpad) return;
    const double *a = (b < n) ? reqs[b].a64 : nullptr;
    double mx = 0.0;
    for (int k = lane; k < N; k += 32) mx = fmax(mx, fabs(a ? a[k] : 0.0));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
    const double inv = ldexp(1.0, -e);
    for (int k = lane; k < Kp; k += 32) {
        uint16_t s[kS];
        slice8((a && k < N) ? a[k] * inv : 0.0, s);
#pragma unroll
        for (int p = 0; p < kS; p++) A[((size_t)p * Bpad + b) * Kp + k] = s[p];
    }
    if (lane == 0) sa[b] = ldexpf(1.0f, e);
}

// Basis slices, one thread per column (t, l, q): T_p[col][n] and 2^(eT - 16 - 8(S-1)).
__global__ void k_basis_slices(const double *__restrict__ T, int L, int N, int Q, int Kp, uint16_t *Tsl, float *scT)
{
    const size_t ncol = (size_t)3 * L * Q;
    for (size_t col = (size_t)blockIdx.x * blockDim.x + threadIdx.x; col < ncol;
         col += (size_t)gridDim.x * blockDim.x) {
        const size_t tl = col / Q, q = col % Q;
        const double *src = T + tl * (size_t)N * Q + q;
        double mx = 0.0;
        for (int k = 0; k < N; k++) mx = fmax(mx, fabs(src[(size_t)k * Q]));
        int e = 0;
        if (mx > 0.0) frexp(mx, &e);
        const double inv = ldexp(1.0, -e);
        for (int k = 0; k < Kp; k++) {
            uint16_t s[kS];
            slice8(k < N ? src[(size_t)k * Q] * inv : 0.0, s);
#pragma unroll
            for (int p = 0; p < kS; p++) Tsl[((size_t)p * ncol + col) * Kp + k] = s[p];
        }
        scT[col] = (mx > 0.0) ? (float)ldexp(1.0, e - 16 - 8 * (kS - 1)) : 0.0f;
    }
}

// ---------------------------------------------------------------- main kernel
struct TcArgs {
    const ReqDev *reqs;
    int n, Bpad, nbt, nqt, n_esel, L, Q, Rn, RT, MT;
    const int *esel;
    const float *scT;    // [3][L][Q]
    const float *sa;     // [Bpad]
    float *Y;            // [3][n_esel][X][RT][MT][n]  (cosmology fastest)
    int *err;            // host-mapped error word
};

__global__ void __launch_bounds__(kThreads, 1)
k_contract_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs args)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment for the swizzled tiles
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = smem;                                  // kS x 16 KB
    unsigned char *sB = smem + kS * kASliceBytes;              // kStages x kS x 4 KB
    uint64_t *bars = (uint64_t *)(sB + kStages * kBStageBytes);
    uint64_t *full = bars, *empty = bars + kStages, *afull = bars + 2 * kStages;
    uint64_t *tfull = afull + 1, *tempty = tfull + 2;
    uint32_t *tmem_slot = (uint32_t *)(tempty + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int btile = blockIdx.x % args.nbt;
    const int n_iter_unit = 3 * args.n_esel;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; i++) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        mbar_init(afull, 1);
        for (int i = 0; i < 2; i++) { mbar_init(&tfull[i], 1); mbar_init(&tempty[i], 128); }
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
        // ------------------------------------------------ TMA producer (whole warp waits, lane 0 issues)
        if (lane == 0) {
            mbar_expect_tx(afull, kS * kASliceBytes);
            tma_load_3d(sA, &mapA, afull, 0, btile * kM, 0);
        }
        uint32_t g = 0;
        bool ok = true;
        for (int u = blockIdx.x; ok && u < args.nbt * args.nqt; u += gridDim.x) {
            const int q0 = (u / args.nbt) * kQT;
            for (int it = 0; it < n_iter_unit; it++, g++) {
                const int st = g % kStages;
                const uint32_t ph = (g / kStages) & 1;
                if (*abort_flag || !mbar_wait(&empty[st], ph ^ 1)) {
                    if (lane == 0) { atomicExch(args.err, 1); *abort_flag = 1; }
                    ok = false;
                    break;
                }
                if (lane == 0) {
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
            mbar_wait(&full[h % kStages], (h / kStages) & 1);
        mbar_wait(afull, 0);
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (whole warp waits, lane 0 issues)
        bool ok = mbar_wait(afull, 0);
        if (!ok && lane == 0) { atomicExch(args.err, 2); *abort_flag = 1; }
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        uint32_t g = 0;
        for (int u = blockIdx.x; ok && u < args.nbt * args.nqt; u += gridDim.x) {
            for (int it = 0; it < n_iter_unit; it++, g++) {
                const int st = g % kStages;
                const uint32_t ph = (g / kStages) & 1;
                const int buf = g & 1;
                const uint32_t tph = (g >> 1) & 1;
                if (*abort_flag || !mbar_wait(&full[st], ph) || !mbar_wait(&tempty[buf], tph ^ 1)) {
                    if (lane == 0) { atomicExch(args.err, 3); *abort_flag = 1; }
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (lane == 0) {
                    const uint32_t dbase = tmem + buf * (kS * kQT);
                    const uint32_t bst = b0 + st * kBStageBytes;
#pragma unroll
                    for (int lev = 0; lev < kS; lev++) {
#pragma unroll
                        for (int p = 0; p <= lev; p++) {
                            const int q = lev - p;
#pragma unroll
                            for (int kk = 0; kk < kKC / 16; kk++) {
                                const uint64_t ad = sdesc(a0 + p * kASliceBytes + kk * 32);
                                const uint64_t bd = sdesc(bst + q * kBSliceBytes + kk * 32);
                                umma(dbase + lev * kQT, ad, bd, (p > 0 || kk > 0) ? 1u : 0u);
                            }
                        }
                    }
                    umma_commit(&empty[st]);
                    umma_commit(&tfull[buf]);
                }
                __syncwarp();
            }
        }
    } else {
        // ------------------------------------------------ epilogue: one cosmology per thread
        const int quad = warp & 3;
        const int bl_ = quad * 32 + lane;
        const int b = btile * kM + bl_;
        const bool valid = b < args.n;
        const ReqDev *rq = valid ? &args.reqs[b] : nullptr;
        const int ng = valid ? rq->n_clust : 0, ns = valid ? rq->n_lens : 0;
        const float sa = args.sa[b < args.Bpad ? b : 0];
        const uint32_t lane_addr = ((uint32_t)(quad * 32)) << 16;
        uint32_t g = 0;
        bool ok = true;
        for (int u = blockIdx.x; ok && u < args.nbt * args.nqt; u += gridDim.x) {
            const int q0 = (u / args.nbt) * kQT;
            const int a = q0 / args.Rn, rt = (q0 % args.Rn) / kQT;
            float wv[kNB][kQT];
            for (int t = 0; t < 3 && ok; t++) {
                const int offB = (t == 0) ? 0 : ng, nB = (t == 0) ? ng : ns;
                if (t < 2) {
#pragma unroll
                    for (int j = 0; j < kNB; j++) {
                        const float4 *src = (valid && j < nB)
                                                ? reinterpret_cast<const float4 *>(rq->V32 + (size_t)(offB + j) * args.Q + q0)
                                                : nullptr;
#pragma unroll
                        for (int c = 0; c < kQT / 4; c++) {
                            float4 v = src ? src[c] : make_float4(0.f, 0.f, 0.f, 0.f);
                            wv[j][4 * c] = v.x; wv[j][4 * c + 1] = v.y; wv[j][4 * c + 2] = v.z; wv[j][4 * c + 3] = v.w;
                        }
                    }
                }
                for (int es = 0; es < args.n_esel; es++, g++) {
                    const int buf = g & 1;
                    const uint32_t tph = (g >> 1) & 1;
                    if (!mbar_wait(&tfull[buf], tph)) { atomicExch(args.err, 4); ok = false; break; }
                    tc_fence_after();
                    const int e = args.esel[es];
                    const float *sc = args.scT + ((size_t)t * args.L + e) * args.Q + q0;
                    float Yj[kNB];
#pragma unroll
                    for (int j = 0; j < kNB; j++) Yj[j] = 0.f;
#pragma unroll
                    for (int c0 = 0; c0 < kQT; c0 += 4) {
                        uint32_t D[kS][4];
#pragma unroll
                        for (int lev = 0; lev < kS; lev++)
                            tmem_ld4(tmem + lane_addr + buf * (kS * kQT) + lev * kQT + c0, D[lev]);
                        tmem_wait_ld();
#pragma unroll
                        for (int c = 0; c < 4; c++) {
                            long long W = (long long)__float2int_rn(__uint_as_float(D[0][c]));
#pragma unroll
                            for (int lev = 1; lev < kS; lev++)
                                W = W * 256 + (long long)__float2int_rn(__uint_as_float(D[lev][c]));
                            const float w = (__ll2float_rn(W) * sa) * __ldg(sc + c0 + c);
#pragma unroll
                            for (int j = 0; j < kNB; j++) Yj[j] = fmaf(wv[j][c0 + c], w, Yj[j]);
                        }
                    }
                    tc_fence_before();
                    mbar_arrive(&tempty[buf]);
                    if (valid) {
                        float *y = args.Y + ((((size_t)t * args.n_esel + es) * (args.Q / args.Rn) + a) * args.RT + rt) *
                                                (size_t)args.MT * args.n + b;
#pragma unroll
                        for (int j = 0; j < kNB; j++)
                            if (j < args.MT) y[(size_t)j * args.n] = Yj[j];
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

// Sum over R-tiles and chi nodes for the tensor-core path, FP32, one thread per
// (cosmology, type, ell, B-side tracer j) accumulating every A-side tracer i:
//   C_ij(l) = N_AB(l) sum_a U_i(a) sum_rt Y(t, l, a, rt, j)
__global__ void k_reduce_tc(const ReqDev *__restrict__ reqs, const float *__restrict__ Y, int n, int X, int L,
                            const int *__restrict__ esel, int n_esel, int RT, int MT, const double *__restrict__ pref)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y % MT, es = blockIdx.y / MT, t = blockIdx.z;
    if (b >= n) return;
    const ReqDev &rq = reqs[b];
    const int ng = rq.n_clust, ns = rq.n_lens;
    const int nA = (t == 2) ? ns : ng, nB = (t == 0) ? ng : ns, offA = (t == 2) ? ng : 0;
    if (j >= nB || nA == 0) return;
    const int e = esel[es];
    const int col = rq.e_out[e];
    if (col < 0) return;
    float Z[kMaxTr];
#pragma unroll
    for (int i = 0; i < kMaxTr; i++) Z[i] = 0.f;
    const float *Yp = Y + ((size_t)t * n_esel + es) * (size_t)X * RT * MT * n + (size_t)j * n + b;
    for (int a = 0; a < X; a++) {
        float s = 0.f;
        for (int rt = 0; rt < RT; rt++) s += Yp[((size_t)a * RT + rt) * MT * n];
#pragma unroll
        for (int i = 0; i < kMaxTr; i++)
            if (i < nA) Z[i] = fmaf(rq.U32[(size_t)(offA + i) * X + a], s, Z[i]);
    }
    const double pf = pref[t * L + e];
    const int ngg = ng * (ng + 1) / 2, ngs = ng * ns;
    for (int i = 0; i < nA; i++) {
        int p;
        if (t == 0) { if (i > j) continue; p = i * ng - i * (i - 1) / 2 + (j - i); }
        else if (t == 1) p = ngg + i * ns + j;
        else { if (i > j) continue; p = ngg + ngs + i * ns - i * (i - 1) / 2 + (j - i); }
        double out = pf * (double)Z[i];
        if (rq.status) out = nan("");
        rq.cl[(size_t)p * rq.n_sel + col] = out;
    }
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

size_t tc_smem_bytes() { return 1024 + kS * kASliceBytes + kStages * kBStageBytes + 256; }

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
    if ((rc = ws.tc.ensure((size_t)kS * Bpad * p->Kp * 2 + (size_t)Bpad * 4 + 256))) return rc;
    uint16_t *A = ws.tc.as<uint16_t>();
    float *sa = reinterpret_cast<float *>(A + (size_t)kS * Bpad * p->Kp);
    k_coef_slices<<<Bpad / 8, 256, 0, s>>>(dreq, n, p->N, p->Kp, Bpad, A, sa);
    BL_CUDA(cudaGetLastError());

    CUtensorMap mapA, mapB;
    if ((rc = make_map(&mapA, A, p->Kp, Bpad, kM))) return rc;
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
    k_contract_tc<<<grid, kThreads, smem, s>>>(mapA, mapB, args);
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}

int launch_reduce_tc(blast_plan *p, ReqDev *dreq, int n, const int *d_esel, int n_esel, const void *ypart,
                     cudaStream_t s)
{
    dim3 grid((n + 127) / 128, n_esel * p->max_tr, 3);
    k_reduce_tc<<<grid, 128, 0, s>>>(dreq, (const float *)ypart, n, p->X, p->L, d_esel, n_esel, p->Rn / kQT,
                                     p->max_tr, p->d_pref);
    BL_CUDA(cudaGetLastError());
    return BLAST_OK;
}
