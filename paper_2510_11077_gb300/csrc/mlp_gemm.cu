// BF16 tensor-core GEMM for sm_103a: C[m][n] = sum_k A[m][k] B[n][k], FP32
// accumulation, fused epilogues for the surrogate network's layers.
//
// One CTA = 4 warps = one 128 x BN tile of C with the whole K (<= 256) of the
// tile staged at once:
//   1. thread 0 issues TMA loads of the A and B tiles (K-major, 128-byte
//      swizzle, one 64-element K-atom per load) onto one mbarrier;
//   2. thread 0 issues K/16 tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M=128,
//      N=BN) into a TMEM accumulator and commits them to a second mbarrier;
//   3. all four warps read the accumulator (warp w owns TMEM lanes 32w..32w+31,
//      i.e. rows 32w..32w+31) with tcgen05.ld and apply the epilogue.
// Every wait is bounded by the global timer: on timeout the kernel records an
// error code, waits once more (bounded) for its own copies or MMAs in flight,
// releases its TMEM and returns.
#include <cstdio>

#include <cudaTypedefs.h>

#include "mlp_internal.cuh"

namespace argus {

namespace {

constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s bound on any wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait on an mbarrier phase; records `code` in *err on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
    const uint64_t t0 = globaltimer();
    while (!mbar_try(bar, parity)) {
        if (globaltimer() - t0 > kWaitNs) {
            if (err) atomicExch(err, code);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major tile, 128-byte swizzle, 8-row
// groups 1024 bytes apart (the layout a 128-byte-swizzled TMA box produces).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = uint64_t((addr & 0x3FFFFu) >> 4);
    d |= uint64_t(1) << 16;             // leading byte offset (unused for swizzled K-major)
    d |= uint64_t(1024 >> 4) << 32;     // stride byte offset: next 8-row group
    d |= uint64_t(1) << 46;             // descriptor version for tcgen05
    d |= uint64_t(2) << 61;             // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32"
        " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float gelu_f(float z) {
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
           z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

template <int EPI>
__device__ __forceinline__ void epilogue(const GemmEpiArgs& e, int row, int col0, int z,
                                         float (&v)[16]) {
    if (EPI == kEpiF32) {
        float* o = e.out_f32 + z * e.chunk_stride + int64_t(row) * e.ldo + col0;
        float4* o4 = reinterpret_cast<float4*>(o);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float4 w;
            w.x = v[4 * q + 0] + (e.bias ? e.bias[col0 + 4 * q + 0] : 0.0f);
            w.y = v[4 * q + 1] + (e.bias ? e.bias[col0 + 4 * q + 1] : 0.0f);
            w.z = v[4 * q + 2] + (e.bias ? e.bias[col0 + 4 * q + 2] : 0.0f);
            w.w = v[4 * q + 3] + (e.bias ? e.bias[col0 + 4 * q + 3] : 0.0f);
            o4[q] = w;
        }
        return;
    }
    float d[16];
    if (EPI == kEpiGelu) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float zz = v[j] + e.bias[col0 + j];
            v[j] = zz;
            d[j] = gelu_f(zz);
        }
        if (e.out_f32) {
            float4* o4 = reinterpret_cast<float4*>(e.out_f32 + int64_t(row) * e.ldo + col0);
#pragma unroll
            for (int q = 0; q < 4; ++q) o4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
    } else {   // kEpiGeluBwd
        const float* zr = e.zin + int64_t(row) * e.ldz + col0;
#pragma unroll
        for (int j = 0; j < 16; ++j) d[j] = v[j] * gelu_grad_f(zr[j]);
        if (e.out_f32) {
            float4* o4 = reinterpret_cast<float4*>(e.out_f32 + int64_t(row) * e.ldo + col0);
#pragma unroll
            for (int q = 0; q < 4; ++q) o4[q] = make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
        }
    }
    __nv_bfloat16 hb[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) hb[j] = __float2bfloat16_rn(d[j]);
    if (e.out_bf16) {
        uint4* o = reinterpret_cast<uint4*>(e.out_bf16 + int64_t(row) * e.ldb + col0);
        o[0] = *reinterpret_cast<const uint4*>(&hb[0]);
        o[1] = *reinterpret_cast<const uint4*>(&hb[8]);
    }
    if (e.out_bf16_t) {
#pragma unroll
        for (int j = 0; j < 16; ++j) e.out_bf16_t[int64_t(col0 + j) * e.ldt + row] = hb[j];
    }
}

template <int EPI, int BN>
__global__ void __launch_bounds__(128, 1) k_gemm_tc(const __grid_constant__ CUtensorMap ta,
                                                    const __grid_constant__ CUtensorMap tb, int K,
                                                    GemmEpiArgs e, int* err) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    constexpr uint32_t kCols = BN <= 32 ? 32u : (BN <= 64 ? 64u : (BN <= 128 ? 128u : 256u));
    __shared__ uint32_t s_tmem;
    __shared__ int s_ok;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const int atoms = K / 64;
    const uint32_t sA = base;
    const uint32_t sB = base + uint32_t(atoms) * (kGemmM * 128u);
    const uint32_t bar_load = sB + uint32_t(atoms) * (BN * 128u);
    const uint32_t bar_mma = bar_load + 8u;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * kGemmM, n0 = blockIdx.y * BN, kz = blockIdx.z * K;

    if (tid == 0) {
        mbar_init(bar_load, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    bool issued = false;
    if (tid == 0) {
        mbar_expect_tx(bar_load, uint32_t(atoms) * (kGemmM + BN) * 128u);
        for (int a = 0; a < atoms; ++a) {
            tma_load_2d(sA + uint32_t(a) * (kGemmM * 128u), &ta, kz + a * 64, m0, bar_load);
            tma_load_2d(sB + uint32_t(a) * (BN * 128u), &tb, kz + a * 64, n0, bar_load);
        }
        if (mbar_wait(bar_load, 0, err, 1)) {
            tc_fence_after();
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                   ((uint32_t(BN) >> 3) << 17) | ((uint32_t(kGemmM) >> 4) << 24);
            for (int k = 0; k < K / 16; ++k) {
                const uint32_t a = uint32_t(k >> 2), kk = uint32_t(k & 3);
                const uint64_t da = smem_desc(sA + a * (kGemmM * 128u) + kk * 32u);
                const uint64_t db = smem_desc(sB + a * (BN * 128u) + kk * 32u);
                tc_mma(tmem, da, db, idesc, k > 0 ? 1u : 0u);
            }
            tc_commit(bar_mma);
            issued = true;
        } else {
            s_ok = 0;
            mbar_wait(bar_load, 0, nullptr, 0);   // let copies in flight land (bounded)
        }
    }
    __syncthreads();
    if (s_ok) {
        if (mbar_wait(bar_mma, 0, err, 2)) {
            tc_fence_after();
            const int row = m0 + tid;
            const uint32_t lane_base = tmem + (uint32_t(warp * 32) << 16);
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                tmem_ld16(lane_base + uint32_t(c0), v);
                epilogue<EPI>(e, row, n0 + c0, blockIdx.z, v);
            }
        } else if (issued) {
            mbar_wait(bar_mma, 0, nullptr, 0);    // let MMAs in flight finish (bounded)
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                     : "memory");
    }
}

template <int EPI, int BN>
cudaError_t launch_one(const CUtensorMap* ta, const CUtensorMap* tb, int M, int N, int K, int chunks,
                       const GemmEpiArgs& e, int* err, cudaStream_t s) {
    const size_t smem = 1024 + size_t(K / 64) * (kGemmM + BN) * 128 + 64;
    static bool configured[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !configured[dev]) {
        const size_t max_smem = 1024 + size_t(kGemmKMax / 64) * (kGemmM + BN) * 128 + 64;
        cudaError_t ce = cudaFuncSetAttribute(k_gemm_tc<EPI, BN>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              int(max_smem));
        if (ce != cudaSuccess) return ce;
        configured[dev] = true;
    }
    dim3 grid(M / kGemmM, N / BN, chunks);
    k_gemm_tc<EPI, BN><<<grid, 128, smem, s>>>(*ta, *tb, K, e, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_tc(const CUtensorMap* ta, const CUtensorMap* tb, int M, int N, int K,
                           int bn, int chunks, int epi, const GemmEpiArgs& e, int* err,
                           cudaStream_t s) {
    if (M <= 0 || M % kGemmM || K <= 0 || K % 64 || K > kGemmKMax || chunks < 1 ||
        (bn != 64 && bn != 128) || N % bn)
        return cudaErrorInvalidValue;
    if (epi != kEpiF32 && (N % 16)) return cudaErrorInvalidValue;
    switch (epi * 1000 + bn) {
        case kEpiF32 * 1000 + 64: return launch_one<kEpiF32, 64>(ta, tb, M, N, K, chunks, e, err, s);
        case kEpiF32 * 1000 + 128: return launch_one<kEpiF32, 128>(ta, tb, M, N, K, chunks, e, err, s);
        case kEpiGelu * 1000 + 64: return launch_one<kEpiGelu, 64>(ta, tb, M, N, K, chunks, e, err, s);
        case kEpiGelu * 1000 + 128: return launch_one<kEpiGelu, 128>(ta, tb, M, N, K, chunks, e, err, s);
        case kEpiGeluBwd * 1000 + 64: return launch_one<kEpiGeluBwd, 64>(ta, tb, M, N, K, chunks, e, err, s);
        case kEpiGeluBwd * 1000 + 128: return launch_one<kEpiGeluBwd, 128>(ta, tb, M, N, K, chunks, e, err, s);
    }
    return cudaErrorInvalidValue;
}

bool make_tmap_bf16(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols,
                    uint32_t box_rows) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || (cols * 2) % 16 || cols % 64 || box_rows > 256)
        return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {64, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace argus
