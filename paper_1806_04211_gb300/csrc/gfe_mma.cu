// Block multiply-add C := W + A B (mod p) on the 5th-generation tensor cores
// (the job MAD of arXiv 1806.04211, Section 4.1; the dominant cost of the
// method, Section 5).
//
// Operands are stored as centred residues: e4m3 for p <= 31 (|c| <= 15,
// tcgen05.mma kind::f8f6f4) or bf16 (|c| <= 125, kind::f16), both with fp32
// accumulation in TMEM.  The MMA is exact as
// long as every partial sum is an integer below 2^24 in magnitude, so the
// host splits K into chunks of at most (2^24 - 1) / cmax^2 (cmax = the
// largest centred magnitude, (p-1)/2, or 1 for GF(2)); each chunk's result
// is reduced mod p in the epilogue on integers.  This is the floating-point
// representation of field elements the paper cites as prior art (Section 1)
// with the exact integer reduction done here.
//
// Kernel (persistent, one CTA of 320 threads per SM, 128 x 256 tiles):
//   warp 0 lane 0 : TMA producer (A tile 128 rows x 128 B of K, K-major,
//                   128B swizzle; B as 128-byte-wide MN-major slabs)
//   warp 1 lane 0 : MMA issuer (4 x tcgen05.mma M128 N256, 32 bytes of K
//                   each, per stage) into one of two TMEM accumulators
//   warps 2..9    : epilogue, warp w reads TMEM lanes 32(w%4).. and one half
//                   of the columns; reduces mod p in fp32 (exact below 2^24),
//                   adds W and packs with cvt to e4m3x2 / bf16x2
// Four pipeline stages with full/empty mbarriers and two accumulator
// full/empty pairs; every wait is bounded by a %globaltimer limit after
// which the CTA records an error, frees its TMEM and returns.
#include "gfe_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

namespace gfe {

namespace {

constexpr int TBM = 128, TBN = 256, TSTAGES = 4;

// Per element width: a stage holds 128 bytes of K per row (64 bf16 or 128
// e4m3), one MMA instruction consumes 32 bytes of K (16 bf16 or 32 e4m3), and
// B arrives as 128-byte-wide MN-major slabs (64 or 128 columns).
template <bool F8> struct Cfg {
    static constexpr int ES = F8 ? 1 : 2;
    static constexpr int TBK = 128 / ES;
    static constexpr int KPI = 32 / ES;
    static constexpr int SLAB_N = 128 / ES;
    static constexpr int NSLAB = TBN / SLAB_N;
    static constexpr int A_STAGE = TBM * 128;        // 16 KB
    static constexpr int B_SLAB = TBK * 128;         // TBK K-rows x 128 B
    static constexpr int B_STAGE = NSLAB * B_SLAB;   // 32 KB
    // instruction descriptor: D f32; A, B bf16 (kind::f16) or e4m3
    // (kind::f8f6f4); A K-major, B MN-major; N = 256, M = 128
    static constexpr uint32_t IDESC = (1u << 4) | ((F8 ? 0u : 1u) << 7) | ((F8 ? 0u : 1u) << 10) | (0u << 15) |
                                      (1u << 16) | ((uint32_t)(TBN >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);
};
constexpr int TC_SMEM = TSTAGES * (Cfg<false>::A_STAGE + Cfg<false>::B_STAGE) + 1024 + 256;
constexpr int TBK = 64;  // K granule that keeps chunk offsets 16-byte aligned for both widths
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false (and *err set) after WAIT_NS
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, int *err) {
    if (mbar_test(b, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_test(b, parity)) {
        if (gtimer() - t0 > WAIT_NS) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// shared-memory matrix descriptor (tcgen05): start, leading / stride byte
// offsets, version 1, 128-byte swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// mod p of an exactly integer-valued float |x| < 2^24: the quotient from the
// reciprocal is off by at most one and the fma residual is exact
__device__ __forceinline__ float fmodp(float x, float pf, float invp) {
    const float q = floorf(x * invp);
    float r = fmaf(-q, pf, x);
    r = r < 0.f ? r + pf : r;
    return r >= pf ? r - pf : r;
}

__device__ __forceinline__ uint32_t pack_e4m3x2(float lo, float hi) {
    uint16_t d;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ void unpack_e4m3x2(uint32_t two, float &lo, float &hi) {
    uint32_t h2;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"((uint16_t)two));
    lo = __half2float(__ushort_as_half((unsigned short)(h2 & 0xFFFF)));
    hi = __half2float(__ushort_as_half((unsigned short)(h2 >> 16)));
}

constexpr int TC_THREADS = 320;  // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr int EPI_WARPS = 8;

// Tile order: bands of TBAND columns of tiles; within a band, TBAND tiles
// of one row of tiles after another.  The tiles resident at the same time
// (about one per SM) then cover a block of about (SMs / TBAND) x TBAND
// tiles, whose A rows and B columns both stay in L2.  (With the rows of
// tiles fastest, A would be read from HBM once per 256 columns: for the
// ClearUp products of Step 3, whose A has tens of thousands of rows, that
// made the kernel HBM-bound.)
constexpr int TBAND = 8;
__device__ __forceinline__ void tile_of(int t, int mt, int nt, int &m0, int &n0) {
    const int band = t / (mt * TBAND);
    const int idx = t - band * mt * TBAND;
    const int w = min(TBAND, nt - band * TBAND);
    m0 = (idx / w) * TBM;
    n0 = (band * TBAND + idx % w) * TBN;
}

// Persistent: CTA c handles tiles c, c + gridDim.x, ... in the order of
// tile_of.  The accumulator is double-buffered in TMEM (2 x 256 fp32
// columns) so the epilogue of one tile overlaps the MMAs of the next.
template <bool F8>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_mad_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int p, int M,
             int N, int K, const void *Wv, int64_t ldw, void *Cv, int64_t ldc, int *err, uint64_t *tslot) {
    using G = Cfg<F8>;
    constexpr int TBK = G::TBK, A_STAGE = G::A_STAGE, B_STAGE = G::B_STAGE, B_SLAB = G::B_SLAB;
    extern __shared__ __align__(1024) uint8_t smraw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = sm;
    uint8_t *sB = sm + TSTAGES * A_STAGE;
    uint64_t *bars = (uint64_t *)(sm + TSTAGES * (A_STAGE + B_STAGE));
    uint64_t *full = bars, *empty = bars + TSTAGES;
    uint64_t *accf = bars + 2 * TSTAGES, *acce = bars + 2 * TSTAGES + 2;
    __shared__ uint32_t tmem_base;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // launch trace: the first CTA to start stamps the start, the last to end
    // the end (%globaltimer, ns); slot = {start, end, CTAs in, CTAs out}
    if (tslot && threadIdx.x == 0 && atomicAdd((unsigned long long *)&tslot[2], 1ull) == 0ull) tslot[0] = gtimer();
    const int mt = (M + TBM - 1) / TBM, nt = (N + TBN - 1) / TBN;
    const int ntiles = mt * nt;
    const int nk = (K + TBK - 1) / TBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TSTAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * TBN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ---- TMA producer (one lane) ----
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                int m0, n0;
                tile_of(t, mt, nt, m0, n0);
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = it % TSTAGES;
                    const uint32_t ph = (uint32_t)(it / TSTAGES) & 1u;
                    if (it >= TSTAGES && !mbar_wait(&empty[s], ph ^ 1u, err)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[s], A_STAGE + B_STAGE);
                    tma_load_2d(sA + s * A_STAGE, &mapA, kb * TBK, m0, &full[s]);
#pragma unroll
                    for (int q = 0; q < G::NSLAB; ++q)
                        tma_load_2d(sB + s * B_STAGE + q * B_SLAB, &mapB, n0 + G::SLAB_N * q, kb * TBK, &full[s]);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer (one lane) ----
        if (lane == 0) {
            int it = 0, i = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
                const int b = i & 1;
                const uint32_t use = (uint32_t)(i >> 1);
                if (i >= 2 && !mbar_wait(&acce[b], (use & 1u) ^ 1u, err)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(b * TBN);
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = it % TSTAGES;
                    const uint32_t ph = (uint32_t)(it / TSTAGES) & 1u;
                    if (!mbar_wait(&full[s], ph, err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(sA + s * A_STAGE), b0 = smem_u32(sB + s * B_STAGE);
#pragma unroll
                    for (int kk = 0; kk < TBK / G::KPI; ++kk) {
                        const uint64_t ad = sdesc(a0 + kk * 32, 16, 1024);
                        const uint64_t bd = sdesc(b0 + kk * G::KPI * 128, B_SLAB, 1024);
                        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                        if constexpr (F8)
                            asm volatile(
                                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                                "l"(ad), "l"(bd), "r"(G::IDESC), "r"(acc));
                        else
                            asm volatile(
                                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                                "l"(ad), "l"(bd), "r"(G::IDESC), "r"(acc));
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&empty[s]))
                                 : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&accf[b]))
                             : "memory");
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: 8 warps; warp w reads TMEM lanes 32*(w%4).. and one
        //      half (128 columns) of the 256-column accumulator ----
        const int e = warp - 2;
        const int quarter = warp & 3, half = e >> 2;
        const float pf = (float)p, invp = 1.0f / (float)p, halfp = (float)(p >> 1);
        const bool vec = ((ldc * G::ES) % 16 == 0) && (((uintptr_t)Cv & 15) == 0) &&
                         (!Wv || (((ldw * G::ES) % 16 == 0) && (((uintptr_t)Wv & 15) == 0)));
        // W words of one 32-column chunk: 32 e4m3 bytes or 32 bf16
        constexpr int WQ = F8 ? 2 : 4;
        int i = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
            const int b = i & 1;
            const uint32_t use = (uint32_t)(i >> 1);
            int m0, n0;
            tile_of(t, mt, nt, m0, n0);
            const int row = m0 + quarter * 32 + lane;
            // this thread's W (its row, the warp's 128 columns) is loaded before
            // the accumulator is waited for, so its latency overlaps the MMAs
            uint4 wpre[4][WQ];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int cb = n0 + half * 128 + 32 * q;
                const bool full = Wv && vec && row < M && cb + 32 <= N;
#pragma unroll
                for (int h = 0; h < WQ; ++h)
                    wpre[q][h] = full ? ((const uint4 *)((const char *)Wv + ((int64_t)row * ldw + cb) * G::ES))[h]
                                      : make_uint4(0, 0, 0, 0);
            }
            const bool have = __all_sync(0xffffffffu, mbar_wait(&accf[b], use & 1u, err));
            if (!have) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int qc = 0; qc < 4; ++qc) {
                const int c0 = half * 128 + 32 * qc;
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * TBN + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                    "[%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                      "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                      "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row >= M) continue;
                const int cb = n0 + c0;
                const bool full_chunk = vec && cb + 32 <= N;
                if constexpr (F8) {
                    if (p == 2 && full_chunk) {
                        // GF(2): the codes are 0 and 1.0, so every partial sum is
                        // an integer in [0, 2^22] (the k chunk) and adding 2^23
                        // puts it in the mantissa: its parity is bit 0.  Bytes of
                        // four results gather into one word, W's bit (bit 3 of a
                        // code 0x38) is XORed in, and x 0x38 gives the e4m3 codes.
                        uint32_t o[8];
#pragma unroll
                        for (int g4 = 0; g4 < 8; ++g4) {
                            uint32_t u[4];
#pragma unroll
                            for (int h = 0; h < 4; ++h)
                                u[h] = __float_as_uint(__uint_as_float(v[4 * g4 + h]) + 8388608.0f);
                            const uint32_t lo = __byte_perm(u[0], u[1], 0x0040), hi = __byte_perm(u[2], u[3], 0x0040);
                            uint32_t bits = __byte_perm(lo, hi, 0x5410) & 0x01010101u;
                            if (Wv) {
                                const uint4 &w4 = wpre[qc][g4 >> 2];
                                const uint32_t ww = (g4 & 3) == 0 ? w4.x : (g4 & 3) == 1 ? w4.y : (g4 & 3) == 2 ? w4.z : w4.w;
                                bits ^= (ww >> 3) & 0x01010101u;
                            }
                            o[g4] = bits * 0x38u;
                        }
                        uint4 *cp = (uint4 *)((uint8_t *)Cv + (int64_t)row * ldc + cb);
                        cp[0] = make_uint4(o[0], o[1], o[2], o[3]);
                        cp[1] = make_uint4(o[4], o[5], o[6], o[7]);
                        continue;
                    }
                }
                float x[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) x[j] = fmodp(__uint_as_float(v[j]), pf, invp);
                // + W (centred, |w| <= (p-1)/2), back into [0, p), then centred
                if (Wv) {
                    if (full_chunk) {
                        if constexpr (F8) {
#pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                const uint4 w4 = wpre[qc][q];
                                const uint32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                                for (int h = 0; h < 4; ++h) {
                                    float a0, a1, a2, a3;
                                    unpack_e4m3x2(ww[h] & 0xFFFF, a0, a1);
                                    unpack_e4m3x2(ww[h] >> 16, a2, a3);
                                    x[16 * q + 4 * h] += a0;
                                    x[16 * q + 4 * h + 1] += a1;
                                    x[16 * q + 4 * h + 2] += a2;
                                    x[16 * q + 4 * h + 3] += a3;
                                }
                            }
                        } else {
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const uint4 w4 = wpre[qc][q];
                                const uint32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                                for (int h = 0; h < 4; ++h) {
                                    x[8 * q + 2 * h] += __uint_as_float(ww[h] << 16);
                                    x[8 * q + 2 * h + 1] += __uint_as_float(ww[h] & 0xFFFF0000u);
                                }
                            }
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if (cb + j >= N) continue;
                            if constexpr (F8) {
                                float lo, hi;
                                unpack_e4m3x2(((const uint8_t *)Wv)[(int64_t)row * ldw + cb + j], lo, hi);
                                x[j] += lo;
                            } else {
                                x[j] += __uint_as_float((uint32_t)((const uint16_t *)Wv)[(int64_t)row * ldw + cb + j]
                                                        << 16);
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        float r = x[j];
                        r = r < 0.f ? r + pf : r;
                        x[j] = r >= pf ? r - pf : r;
                    }
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) x[j] = x[j] > halfp ? x[j] - pf : x[j];
                if (full_chunk) {
                    if constexpr (F8) {
                        uint4 *cp = (uint4 *)((uint8_t *)Cv + (int64_t)row * ldc + cb);
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            uint32_t ww[4];
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                const int j = 16 * q + 4 * h;
                                ww[h] = pack_e4m3x2(x[j], x[j + 1]) | (pack_e4m3x2(x[j + 2], x[j + 3]) << 16);
                            }
                            cp[q] = make_uint4(ww[0], ww[1], ww[2], ww[3]);
                        }
                    } else {
                        uint4 *cp = (uint4 *)((uint16_t *)Cv + (int64_t)row * ldc + cb);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            uint32_t ww[4];
#pragma unroll
                            for (int h = 0; h < 4; ++h) ww[h] = pack_bf16x2(x[8 * q + 2 * h], x[8 * q + 2 * h + 1]);
                            cp[q] = make_uint4(ww[0], ww[1], ww[2], ww[3]);
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        if (cb + j >= N) continue;
                        if constexpr (F8)
                            ((uint8_t *)Cv)[(int64_t)row * ldc + cb + j] = (uint8_t)(pack_e4m3x2(x[j], 0.f) & 0xFF);
                        else
                            ((uint16_t *)Cv)[(int64_t)row * ldc + cb + j] = (uint16_t)(pack_bf16x2(x[j], 0.f) & 0xFFFF);
                    }
                }
            }
            // this warp has read its part of accumulator b: release it
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[b])) : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TBN));
    if (tslot && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd((unsigned long long *)&tslot[3], 1ull) == (unsigned long long)gridDim.x - 1) tslot[1] = gtimer();
    }
}

// Failure-detection self-test: waits (with the kernel's bounded-wait helper
// and a caller-given limit) on an mbarrier phase that nothing completes; the
// wait gives up, the error word is set and the kernel returns normally.
__global__ void k_wait_selftest(uint64_t limit_ns, int *err, int *gave_up) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t t0 = gtimer();
        bool ok = false;
        while (!(ok = mbar_test(&bar, 0)) && gtimer() - t0 < limit_ns) {
        }
        if (!ok) {
            atomicExch(err, 1);
            *gave_up = 1;
        }
    }
}

// ---- host side ----
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_once;
std::mutex g_dev_mu;
constexpr int MAX_DEV = 64;
bool g_attr_dev[MAX_DEV] = {};

int g_num_sms = 148;

// per-device set-up with the device current (the kernels' shared-memory
// attribute, the SM count); false on a CUDA error
bool dev_setup() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return false;
    std::lock_guard<std::mutex> g(g_dev_mu);
    if (!g_attr_dev[dev]) {
        if (cudaFuncSetAttribute(k_mad_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_mad_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) != cudaSuccess)
            return false;
        g_attr_dev[dev] = true;
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
            g_num_sms = nsm;
    }
    return true;
}

bool init_tc() {
    std::call_once(g_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_encode != nullptr;
}

// 2-D tensor map of bf16 (es = 2) or byte (es = 1) elements: inner dimension
// `inner` (contiguous), `outer` rows of pitch `ld` elements, box of 128
// bytes x box_outer, 128-byte swizzle, zero fill out of bounds.
bool make_map(CUtensorMap *map, const void *base, int64_t inner, int64_t outer, int64_t ld, int box_outer, int es) {
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                          const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

inline bool al16(const void *p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

// largest K (multiple of 64) whose fp32 partial sums stay exact integers
// GF(2) takes 2^22: its epilogue reads the parity of a partial sum below
// 2^23 from the mantissa of (sum + 2^23)
int64_t tc_k_chunk(int p) {
    if (p == 2) return ((int64_t)1 << 22) / TBK * TBK;
    const int64_t cmax = (p - 1) / 2;
    const int64_t kc = (((int64_t)1 << 24) - 1) / (cmax * cmax);
    return kc / TBK * TBK;
}

bool mad_tc(const Launch &L, int64_t m, int64_t n, int64_t k, const void *W, int64_t ldw, const void *A, int64_t lda,
            const void *B, int64_t ldb, void *C, int64_t ldc) {
    const bool f8 = L.codec == CODEC_F8;
    const int es = f8 ? 1 : 2;
    if (!al16(A) || !al16(B) || (lda * es) % 16 || (ldb * es) % 16) return false;
    if (m > (1 << 30) || n > (1 << 30) || ((m + TBM - 1) / TBM) * ((n + TBN - 1) / TBN) > INT32_MAX) return false;
    // every call passes its own error word; without one the bounded waits
    // could report nowhere, so the shape goes to the CUDA-core path
    int *err = L.err;
    if (!err || !init_tc() || !dev_setup()) return false;
    const int64_t kc = tc_k_chunk(L.p);
    for (int64_t k0 = 0; k0 < k; k0 += kc) {
        const int64_t kk = k - k0 < kc ? k - k0 : kc;
        const char *Ak = (const char *)A + k0 * es;
        const char *Bk = (const char *)B + k0 * ldb * es;
        CUtensorMap ma, mb;
        if (!make_map(&ma, Ak, kk, m, lda, TBM, es) || !make_map(&mb, Bk, n, kk, ldb, 128 / es, es)) {
            if (k0 == 0) return false;  // nothing launched yet: the caller takes the plain path
            mad_plain(L, m, n, k - k0, C, ldc, Ak, lda, Bk, ldb, C, ldc);
            return true;
        }
        const void *Wk = k0 ? C : W;
        const int64_t ldwk = k0 ? ldc : ldw;
        const int64_t tiles = ((m + TBM - 1) / TBM) * ((n + TBN - 1) / TBN);
        int64_t ctas = g_num_sms;
        if (L.tiles_per_cta > 0) ctas = std::max<int64_t>(ctas, (tiles + L.tiles_per_cta - 1) / L.tiles_per_cta);
        const unsigned grid = (unsigned)(tiles < ctas ? tiles : ctas);
        // timed on the device when the launch trace has a slot, else by events
        uint64_t *tslot = prof_device_slot(L, K_MAD_TC, m, n, kk);
        cudaEvent_t ev = nullptr;
        if (!tslot) prof_begin(L, K_MAD_TC, &ev);
        else prof_count(K_MAD_TC);
        if (f8)
            k_mad_tc<true><<<grid, TC_THREADS, TC_SMEM, L.st>>>(ma, mb, L.p, (int)m, (int)n, (int)kk, Wk, ldwk, C,
                                                                ldc, err, tslot);
        else
            k_mad_tc<false><<<grid, TC_THREADS, TC_SMEM, L.st>>>(ma, mb, L.p, (int)m, (int)n, (int)kk, Wk, ldwk, C,
                                                                 ldc, err, tslot);
        prof_end(L, K_MAD_TC, ev, (double)m * (double)n * (double)kk,
                 (double)es * ((double)m * kk + (double)kk * n + (Wk ? 2.0 : 1.0) * (double)m * n), m, n, kk);
    }
    return true;
}

bool read_error_word(cudaStream_t st, const int *err, int *value) {
    *value = 0;
    if (!err) return true;
    // pageable destination: the copy is ordered after the work on st and
    // returns once it is complete
    return cudaMemcpyAsync(value, err, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
           host_wait(st) == cudaSuccess;
}

}  // namespace gfe

namespace gfe {
// launches the self-test on `st` with an error word of its own; returns the
// flag the wait sets when it gives up (or -1 on a CUDA error)
int wait_selftest(cudaStream_t st, int64_t limit_us) {
    int *d = nullptr, h = 0;  // d[0] error word, d[1] gave-up flag
    if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) return -1;
    if (cudaMemsetAsync(d, 0, 2 * sizeof(int), st) != cudaSuccess) {
        cudaFree(d);
        return -1;
    }
    k_wait_selftest<<<1, 32, 0, st>>>((uint64_t)limit_us * 1000ull, d, d + 1);
    const bool ok = cudaMemcpyAsync(&h, d + 1, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                    cudaStreamSynchronize(st) == cudaSuccess;
    cudaFree(d);
    return ok ? h : -1;
}
}  // namespace gfe
