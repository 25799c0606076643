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
// Kernel: one CTA of 128 threads per 128 x 256 tile of C; a stage holds 128
// bytes of K per row (64 bf16 / 128 e4m3).
//   warp 0 lane 0 : TMA producer (A tile 128 rows x 128 B, K-major, 128B
//                   swizzle; B as MN-major slabs 128 B wide)
//   warp 1 lane 0 : MMA issuer (4 x tcgen05.mma M128 N256, 32 bytes of K each)
//   all 4 warps   : epilogue, warp w reads TMEM lanes 32w..32w+31
// Four pipeline stages with full/empty mbarriers; every wait is bounded by a
// %globaltimer limit after which the CTA records an error, frees its TMEM
// and returns.
#include "gfe_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>

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

__device__ __forceinline__ int bf16_int(uint16_t b) { return (int)__uint_as_float((uint32_t)b << 16); }
__device__ __forceinline__ uint16_t int_bf16(int c) { return (uint16_t)(__float_as_uint((float)c) >> 16); }
// e4m3 of a centred residue |c| <= 15 (all such integers are exact in e4m3)
__device__ __forceinline__ int e4m3_int(uint32_t b) {
    const int mag = b & 0x7F;
    if (mag < 0x38) return 0;
    const int v = ((8 + (mag & 7)) << ((mag >> 3) - 7)) >> 3;
    return (b & 0x80) ? -v : v;
}
__device__ __forceinline__ uint32_t int_e4m3(int c) {
    if (c == 0) return 0;
    const int sg = c < 0, a = sg ? -c : c;
    const int e = 31 - __clz(a);
    return (uint32_t)((sg << 7) | ((e + 7) << 3) | (((a << 3) >> e) - 8));
}

// x mod p in [0, p) for |x| < 2^24: the float quotient is off by at most one
__device__ __forceinline__ int modp_f(int x, int p, float invp) {
    const int q = (int)floorf((float)x * invp);
    int r = x - q * p;
    if (r < 0) r += p;
    if (r >= p) r -= p;
    return r;
}
// r in [-(p-1)/2 - p, 2p): the centred representative of r mod p
__device__ __forceinline__ int centre(int r, int p) {
    if (r < 0) r += p;
    if (r >= p) r -= p;
    return r > (p >> 1) ? r - p : r;
}

template <bool F8>
__global__ void __launch_bounds__(128, 1)
    k_mad_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int p, int M,
             int N, int K, const void *Wv, int64_t ldw, void *Cv, int64_t ldc, int *err) {
    using G = Cfg<F8>;
    constexpr int TBK = G::TBK, A_STAGE = G::A_STAGE, B_STAGE = G::B_STAGE, B_SLAB = G::B_SLAB;
    extern __shared__ __align__(1024) uint8_t smraw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = sm;
    uint8_t *sB = sm + TSTAGES * A_STAGE;
    uint64_t *bars = (uint64_t *)(sm + TSTAGES * (A_STAGE + B_STAGE));
    uint64_t *full = bars, *empty = bars + TSTAGES, *accb = bars + 2 * TSTAGES;
    __shared__ uint32_t tmem_base;
    __shared__ int bad;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // M tiles vary fastest: CTAs resident together share the same B columns
    const int m0 = blockIdx.x * TBM, n0 = blockIdx.y * TBN;
    const int nk = (K + TBK - 1) / TBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TSTAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accb, 1);
        bad = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TBN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer ----
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % TSTAGES;
            const uint32_t ph = (uint32_t)(kb / TSTAGES) & 1u;
            if (kb >= TSTAGES && !mbar_wait(&empty[s], ph ^ 1u, err)) {
                bad = 1;
                break;
            }
            mbar_expect_tx(&full[s], A_STAGE + B_STAGE);
            tma_load_2d(sA + s * A_STAGE, &mapA, kb * TBK, m0, &full[s]);
#pragma unroll
            for (int q = 0; q < G::NSLAB; ++q)
                tma_load_2d(sB + s * B_STAGE + q * B_SLAB, &mapB, n0 + G::SLAB_N * q, kb * TBK, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        bool ok = true;
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int s = kb % TSTAGES;
            const uint32_t ph = (uint32_t)(kb / TSTAGES) & 1u;
            if (!mbar_wait(&full[s], ph, err)) {
                ok = false;
                bad = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA + s * A_STAGE), b0 = smem_u32(sB + s * B_STAGE);
#pragma unroll
            for (int kk = 0; kk < TBK / G::KPI; ++kk) {
                // A: K-major, advance 32 bytes of K inside the swizzle atom
                const uint64_t ad = sdesc(a0 + kk * 32, 16, 1024);
                // B: MN-major, KPI K-rows of 128 B further; slabs B_SLAB apart
                const uint64_t bd = sdesc(b0 + kk * G::KPI * 128, B_SLAB, 1024);
                const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                if constexpr (F8)
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(G::IDESC), "r"(acc));
                else
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(G::IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        if (ok)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(accb))
                         : "memory");
    }
    __syncwarp();

    // ---- epilogue: TMEM -> registers -> (+W) mod p -> C ----
    const bool have = __all_sync(0xffffffffu, mbar_wait(accb, 0, err));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (have) {
        const int row = m0 + warp * 32 + lane;
        const float invp = 1.0f / (float)p;
        // 16-byte vector access of W and C when their rows are 16-byte aligned
        const bool vec = ((ldc * G::ES) % 16 == 0) && (((uintptr_t)Cv & 15) == 0) &&
                         (!Wv || (((ldw * G::ES) % 16 == 0) && (((uintptr_t)Wv & 15) == 0)));
#pragma unroll 1
        for (int c0 = 0; c0 < TBN; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
                const int cb = n0 + c0;
                int out[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) out[j] = modp_f((int)__uint_as_float(v[j]), p, invp);
                if (vec && cb + 32 <= N) {
                    if constexpr (F8) {
                        const uint8_t *W = (const uint8_t *)Wv;
                        if (W) {
                            const uint4 *wp = (const uint4 *)(W + (int64_t)row * ldw + cb);
#pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                const uint4 w4 = wp[q];
                                const uint32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                                for (int h = 0; h < 4; ++h)
#pragma unroll
                                    for (int b = 0; b < 4; ++b) out[16 * q + 4 * h + b] += e4m3_int((ww[h] >> (8 * b)) & 0xFF);
                            }
                        }
                        uint4 *cp = (uint4 *)((uint8_t *)Cv + (int64_t)row * ldc + cb);
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            uint32_t ww[4];
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                uint32_t x = 0;
#pragma unroll
                                for (int b = 0; b < 4; ++b) x |= int_e4m3(centre(out[16 * q + 4 * h + b], p)) << (8 * b);
                                ww[h] = x;
                            }
                            cp[q] = make_uint4(ww[0], ww[1], ww[2], ww[3]);
                        }
                    } else {
                        const uint16_t *W = (const uint16_t *)Wv;
                        if (W) {
                            const uint4 *wp = (const uint4 *)(W + (int64_t)row * ldw + cb);
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const uint4 w4 = wp[q];
                                const uint32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                                for (int h = 0; h < 4; ++h) {
                                    out[8 * q + 2 * h] += bf16_int((uint16_t)(ww[h] & 0xFFFF));
                                    out[8 * q + 2 * h + 1] += bf16_int((uint16_t)(ww[h] >> 16));
                                }
                            }
                        }
                        uint4 *cp = (uint4 *)((uint16_t *)Cv + (int64_t)row * ldc + cb);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            uint32_t ww[4];
#pragma unroll
                            for (int h = 0; h < 4; ++h)
                                ww[h] = (uint32_t)int_bf16(centre(out[8 * q + 2 * h], p)) |
                                        ((uint32_t)int_bf16(centre(out[8 * q + 2 * h + 1], p)) << 16);
                            cp[q] = make_uint4(ww[0], ww[1], ww[2], ww[3]);
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = cb + j;
                        if (col < N) {
                            int x = out[j];
                            if constexpr (F8) {
                                if (Wv) x += e4m3_int(((const uint8_t *)Wv)[(int64_t)row * ldw + col]);
                                ((uint8_t *)Cv)[(int64_t)row * ldc + col] = (uint8_t)int_e4m3(centre(x, p));
                            } else {
                                if (Wv) x += bf16_int(((const uint16_t *)Wv)[(int64_t)row * ldw + col]);
                                ((uint16_t *)Cv)[(int64_t)row * ldc + col] = int_bf16(centre(x, p));
                            }
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (bad && threadIdx.x == 0) {
        // drain the TMA loads that may still be in flight (bounded)
        for (int s = 0; s < TSTAGES; ++s) {
            uint64_t t0 = gtimer();
            while (!mbar_test(&full[s], 0) && !mbar_test(&full[s], 1) && gtimer() - t0 < WAIT_NS / 4) {
            }
        }
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TBN));
}

// ---- host side ----
// error word of the kernel: one per device (a module-scope device variable,
// zero at load); its device address is looked up once per device
__device__ int g_tc_err;

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_once;
std::mutex g_dev_mu;
constexpr int MAX_DEV = 64;
int *g_err_dev[MAX_DEV] = {};
bool g_attr_dev[MAX_DEV] = {};

// per-device set-up with the device current; returns the error word
int *dev_setup() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return nullptr;
    std::lock_guard<std::mutex> g(g_dev_mu);
    if (!g_attr_dev[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_tc_err) != cudaSuccess) return nullptr;
        if (cudaFuncSetAttribute(k_mad_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_mad_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) != cudaSuccess)
            return nullptr;
        g_err_dev[dev] = (int *)p;
        g_attr_dev[dev] = true;
    }
    return g_err_dev[dev];
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
int64_t tc_k_chunk(int p) {
    const int64_t cmax = p == 2 ? 1 : (p - 1) / 2;
    const int64_t kc = (((int64_t)1 << 24) - 1) / (cmax * cmax);
    return kc / TBK * TBK;
}

bool mad_tc(const Launch &L, int64_t m, int64_t n, int64_t k, const void *W, int64_t ldw, const void *A, int64_t lda,
            const void *B, int64_t ldb, void *C, int64_t ldc) {
    const bool f8 = L.codec == CODEC_F8;
    const int es = f8 ? 1 : 2;
    if (!al16(A) || !al16(B) || (lda * es) % 16 || (ldb * es) % 16) return false;
    if (m > (1 << 30) || n > ((int64_t)65535 * TBN)) return false;
    if (!init_tc()) return false;
    int *err = dev_setup();
    if (!err) return false;
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
        dim3 grid((unsigned)((m + TBM - 1) / TBM), (unsigned)((n + TBN - 1) / TBN));
        cudaEvent_t ev;
        prof_begin(L, K_MAD_TC, &ev);
        if (f8)
            k_mad_tc<true><<<grid, 128, TC_SMEM, L.st>>>(ma, mb, L.p, (int)m, (int)n, (int)kk, Wk, ldwk, C, ldc, err);
        else
            k_mad_tc<false><<<grid, 128, TC_SMEM, L.st>>>(ma, mb, L.p, (int)m, (int)n, (int)kk, Wk, ldwk, C, ldc, err);
        prof_end(L, K_MAD_TC, ev, (double)m * (double)n * (double)kk);
    }
    return true;
}

int tc_error_flag(bool reset) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return 0;
    int *e = nullptr;
    {
        std::lock_guard<std::mutex> g(g_dev_mu);
        e = g_err_dev[dev];
    }
    if (!e) return 0;
    int h = 0;
    cudaMemcpy(&h, e, sizeof(int), cudaMemcpyDeviceToHost);
    if (reset && h) cudaMemset(e, 0, sizeof(int));
    return h;
}

}  // namespace gfe
