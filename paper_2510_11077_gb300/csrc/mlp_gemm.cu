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

// 32 consecutive columns of this warp's TMEM lanes, one wait
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32"
        " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// GELU and its derivative from e = erf(z / sqrt 2), so that a caller that needs
// both evaluates erf once (the same bits as evaluating each on its own)
__device__ __forceinline__ float erf_gelu(float z) { return erff(z * 0.70710678118654752f); }
__device__ __forceinline__ float gelu_e(float z, float e) { return 0.5f * z * (1.0f + e); }
__device__ __forceinline__ float gelu_grad_e(float z, float e) {
    return 0.5f * (1.0f + e) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}
__device__ __forceinline__ float gelu_f(float z) { return gelu_e(z, erf_gelu(z)); }
__device__ __forceinline__ float gelu_grad_f(float z) { return gelu_grad_e(z, erf_gelu(z)); }

// zpre: for kEpiGeluBwd, the 16 saved pre-activations of these columns when
// the caller loaded them ahead (else NULL: read here)
template <int EPI>
__device__ __forceinline__ void epilogue(const GemmEpiArgs& e, int row, int col0, int z,
                                         float (&v)[16], const float* zpre = nullptr) {
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
        const float* zr = zpre ? zpre : e.zin + int64_t(row) * e.ldz + col0;
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

// 256 threads: thread 0 issues the copies and the MMAs; in the epilogue warps
// w and w + 4 share TMEM lane quadrant w (rows 32w..32w+31), each taking half
// of the tile's columns.
constexpr int kGemmThreads = 256;

template <int EPI, int BN>
__global__ void __launch_bounds__(kGemmThreads, 1) k_gemm_tc(const __grid_constant__ CUtensorMap ta,
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

    // the epilogue's rows and columns; kEpiGeluBwd with 64-column tiles loads
    // its saved pre-activations now, under the copies and the MMAs
    const int quad = warp & 3, half = warp >> 2;
    const int row = m0 + quad * 32 + (tid & 31);
    constexpr int kHalf = BN / 2;
    constexpr bool kPre = EPI == kEpiGeluBwd && BN <= 64;
    float zp[kPre ? kHalf : 1];
    if constexpr (kPre) {
        const float4* z4 = reinterpret_cast<const float4*>(e.zin + int64_t(row) * e.ldz + n0 + half * kHalf);
#pragma unroll
        for (int q = 0; q < kHalf / 4; ++q) {
            const float4 t = z4[q];
            zp[4 * q] = t.x; zp[4 * q + 1] = t.y; zp[4 * q + 2] = t.z; zp[4 * q + 3] = t.w;
        }
    }

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
            const uint32_t lane_base = tmem + (uint32_t(quad * 32) << 16);
#pragma unroll
            for (int c = 0; c < kHalf; c += 16) {
                const int c0 = half * kHalf + c;
                float v[16];
                tmem_ld16(lane_base + uint32_t(c0), v);
                epilogue<EPI>(e, row, n0 + c0, blockIdx.z, v, kPre ? zp + c : nullptr);
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
    k_gemm_tc<EPI, BN><<<grid, kGemmThreads, smem, s>>>(*ta, *tb, K, e, err);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Fused evaluation: a cluster of kCl CTAs (1, 2 or 4; 8 warps each, 16 with 4) owns 128
// rows and runs every layer; CTA rank c of the cluster computes the output
// columns [c N / kCl, (c + 1) N / kCl) of every stage, so that a batch of a few
// thousand rows still spreads over most SMs and each CTA's epilogue (GELU and
// its derivative, the expensive part) is 1/kCl of a layer.
// Shared memory: the 128 x 256 BF16 activation tile (A operand, four 64-column
// K-atoms in the 128-byte-swizzled layout a TMA box would give; two copies
// when kCl > 1, one read by the current stage while the next is filled), this
// rank's weight slice of the current stage (B operand, N / kCl x K, loaded by
// TMA while the previous epilogue runs), biases, the value output's weight
// row, and the rows' quadratic baseline terms.
// Stages (each one tcgen05 GEMM into the CTA's TMEM accumulator):
//   0..3  h_{l+1} = gelu(h_l W_l^T + b_l); gelu'(z) saved for the backward pass
//   4     y = h_4 W_4^T + b_4
//   5..8  (kFusedValueGrad) dz_l = (dz_{l+1} W_l) * gelu'(z_l), then dx = dz_1 W_0,
//         seeded with dz_4 = W_4[0] * gelu'(z_4) (the value output's one-hot)
// After its epilogue each rank writes its columns of the next activation tile
// into its own shared memory, and thread 0 sends them to every other rank
// with bulk copies (cp.async.bulk, shared::cta -> shared::cluster) that
// complete on the receiver's mbarrier of that tile; each rank arms its
// mbarrier with the bytes its peers send and waits on it (bounded) before its
// next MMA, so no cluster-wide barrier sits between stages.  Rank c's columns of a hidden layer are one (kCl = 4) or two
// (kCl = 2) whole K-atoms, contiguous in the tile.  The tiles alternate, so a
// rank writes a tile only after every peer has sent it the next stage's
// columns, which they do only after their MMA has read that tile.  gelu'(z) of
// rank c's columns stays with rank c (the backward stage's column i needs
// layer l's column i): in TMEM behind the accumulator with kCl = 4, else in
// global scratch.  With kCl = 4 the weight slices are double-buffered and
// loaded a stage ahead.  Warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows)
// and column group w / 4 of the rank's columns (16 columns each with 4-CTA
// clusters); gelu'(z) is formed only when the value's gradient is
// back-propagated.  Thread 0 issues the copies and the
// MMAs and alone waits on the mbarriers (bounded); after a timeout the CTA
// stops computing but keeps sending and receiving its tile columns, drains
// its weight copies (bounded), and meets the cluster's one final barrier, so
// no rank waits forever and none exits while a copy into it is in flight.
// The prologue standardizes the inputs (from FP32 theta, or from a sampler's
// FP64 z and centre; every rank builds the whole input tile) and forms the
// quadratic baseline: rank c the terms (H u)_k of the gradient outputs it
// writes and its share of u^T H u, which rank 0 adds up in rank order.
constexpr uint32_t kFAtomA = kGemmM * 128u;       // one 64-column K-atom of the activation tile
constexpr uint32_t kFSmemA = 4u * kFAtomA;        // 64 KB
constexpr int kFBiasFloats = 4 * kMlpHidden + kMlpOutPad;

template <int kCl>
struct FusedCfg {
    // 16 warps with 4-CTA clusters (a rank's 64 columns: 16 per warp); 8 otherwise
    static constexpr int kThreads = kCl == 4 ? 512 : 256;
    static constexpr int kGroups = kThreads / 128;                       // warp groups of 4
    static constexpr int kGc = (256 / kCl) / kGroups;                     // columns per group, 256-wide stage
    static constexpr int kABufs = kCl > 1 ? 2 : 1;
    static constexpr int kBBufs = kCl == 4 ? 2 : 1;                      // weights a stage ahead
    static constexpr uint32_t kSmemB = 4u * (256u / kCl) * 128u;          // 4 K-atoms x N/kCl rows
    static constexpr int kOutCols = kMlpOutPad / kCl;                     // stage 4 and 8 columns
    static constexpr int kGb = (kMlpIn < kOutCols + 1) ? kMlpIn : kOutCols + 1;   // (H u)_k kept
    static constexpr int kTailFloats = kGemmM * kGb + kGemmM * (kCl + 2) + kFBiasFloats + kMlpHidden;
    static constexpr size_t kSmem =
        1024 + kABufs * kFSmemA + kBBufs * kSmemB + sizeof(float) * kTailFloats + 64;
    // gelu'(z) of the four hidden layers: kept in TMEM after the accumulator
    // (columns 64 + 64 l ..) when the rank's 64 columns per layer fit, else in
    // global scratch
    static constexpr bool kGInTmem = kCl == 4;
    static constexpr uint32_t kTmemCols = kGInTmem ? 512u : 256u / kCl;
    static constexpr uint32_t kRankBytes = (256u / kCl) * 128u * 2u;      // a rank's columns of a tile
};

struct FusedStage {
    int map;      // 0..4: maps.w[map]; 5..8: maps.wt[8 - map]
    int K, N;
};
__constant__ FusedStage c_fstage[9] = {{0, kMlpInPad, kMlpHidden}, {1, kMlpHidden, kMlpHidden},
                                       {2, kMlpHidden, kMlpHidden}, {3, kMlpHidden, kMlpHidden},
                                       {4, kMlpHidden, kMlpOutPad}, {5, kMlpHidden, kMlpHidden},
                                       {6, kMlpHidden, kMlpHidden}, {7, kMlpHidden, kMlpHidden},
                                       {8, kMlpHidden, kMlpInPad}};

__device__ __forceinline__ const CUtensorMap* fused_map(const MlpFusedMaps& m, int i) {
    return i < kMlpLayers ? &m.w[i] : &m.wt[8 - i];
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// the address of the same shared-memory offset in cluster CTA `rank`
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// copy `bytes` of this CTA's shared memory to the same offset in cluster CTA
// `rank`, completing on that CTA's mbarrier (at the same offset as bar)
__device__ __forceinline__ void bulk_copy_to_rank(uint32_t src, uint32_t bytes, uint32_t bar,
                                                  uint32_t rank) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            map_rank(src, rank)),
        "r"(src), "r"(bytes), "r"(map_rank(bar, rank))
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
        "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
        "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
        : "memory");
}

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}

// 16 consecutive activations of row r, columns c0..c0+15 (c0 a multiple of 16),
// as BF16 into the swizzled K-major tile at shared address `tile`: 16-byte
// chunk j of a row's 128-byte K-atom row sits at chunk position j ^ (r % 8).
__device__ __forceinline__ void store_act16(uint32_t tile, int r, int c0, const float* d) {
    uint32_t p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(d[2 * i], d[2 * i + 1]);
        p[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    const uint32_t off = tile + uint32_t(c0 >> 6) * kFAtomA + uint32_t(r) * 128u;
    const uint32_t j0 = uint32_t((c0 & 63) >> 3), sw = uint32_t(r & 7);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(off + ((j0 ^ sw) << 4)), "r"(p[0]),
                 "r"(p[1]), "r"(p[2]), "r"(p[3])
                 : "memory");
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(off + (((j0 + 1u) ^ sw) << 4)),
                 "r"(p[4]), "r"(p[5]), "r"(p[6]), "r"(p[7])
                 : "memory");
}

__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// input k of row gr: theta, or float(z - centre) in the FP64-input mode
__device__ __forceinline__ float fused_in(const MlpFusedArgs& a, int64_t gr, int k) {
    return a.z64 ? float(a.z64[gr * kMlpIn + k] - a.zc[k]) : a.theta[gr * kMlpIn + k];
}

// the outputs of row gr: the loglik and, when the mode has one, gradient k
__device__ __forceinline__ void fused_out_ll(const MlpFusedArgs& a, int64_t gr, float ll) {
    if (a.z64) {
        const double v = double(ll) + a.off;
        a.ll64[gr] = isfinite(v) ? v : -INFINITY;
    } else {
        a.loglik[gr] = ll;
    }
}
__device__ __forceinline__ void fused_out_grad(const MlpFusedArgs& a, int64_t gr, int k, float g) {
    if (a.z64) a.g64[gr * kMlpIn + k] = double(g);
    else a.grad[gr * kMlpIn + k] = g;
}

// Trace of one row segment (tests only): `cnt` floats, or their BF16 roundings
// (the values store_act16 writes) with kRound.
template <bool kRound>
__device__ __forceinline__ void trace_row(float* t, int cnt, const float* v) {
#pragma unroll
    for (int j = 0; j < cnt; ++j)
        t[j] = kRound ? __bfloat162float(__float2bfloat16_rn(v[j])) : v[j];
}

// 16 saved gelu'(z) of one row (4 float4), issued early so that their latency
// overlaps other work
__device__ __forceinline__ void load_g16(const float* g, float4 (&o)[4]) {
    const float4* g4 = reinterpret_cast<const float4*>(g);
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = g4[i];
}

// `cnt` (16, 32 or 48) consecutive accumulator columns of this warp's lanes
template <int kCnt>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float (&v)[48]) {
    if (kCnt == 16) {
        float t[16];
        tmem_ld16(taddr, t);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = t[j];
    } else {
        float t[32];
        tmem_ld32(taddr, t);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = t[j];
        if (kCnt == 48) {
            float u[16];
            tmem_ld16(taddr + 32u, u);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[32 + j] = u[j];
        }
    }
}

template <int kCl>
__global__ void __launch_bounds__(FusedCfg<kCl>::kThreads, 1)
    k_mlp_fused(const __grid_constant__ MlpFusedMaps maps, const __grid_constant__ MlpFusedArgs a) {
    using Cfg = FusedCfg<kCl>;
    constexpr int kOut = Cfg::kOutCols;                       // this rank's stage-4/8 columns
    constexpr int kOutLd = kOut > 32 ? 48 : kOut;             // of them read back (<= 48 used)
    constexpr int kBB = Cfg::kBBufs;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ int s_ok;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sB0 = base + Cfg::kABufs * kFSmemA;
    float* tail = reinterpret_cast<float*>(smem_raw + (base - raw) + Cfg::kABufs * kFSmemA +
                                           kBB * Cfg::kSmemB);
    float* gbase_s = tail;                            // [128][kGb]: -(H u)_k, k from k_lo
    float* qpart_s = gbase_s + kGemmM * Cfg::kGb;     // [kCl][128]: each rank's share of u^T H u
    float* y0_s = qpart_s + kGemmM * kCl;             // [128]
    float* spare_s = y0_s + kGemmM;                   // [128]
    float* bias_s = spare_s + kGemmM;                 // b_0..b_3 [256] each, then b_4 [64]
    float* w4_s = bias_s + kFBiasFloats;              // W_4[0] [256]
    // mbarriers: weights (one per B buffer), MMA, and the peers' columns of each A tile
    const uint32_t bar_load0 = smem_u32(w4_s + kMlpHidden);
    const uint32_t bar_mma = bar_load0 + 16u;
    const uint32_t bar_a0 = bar_mma + 8u;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, grp = warp >> 2;                // TMEM lane quarter, column group
    const int r = 32 * q + lane;                            // this thread's row in the slab
    const uint32_t rank = kCl > 1 ? cluster_rank() : 0u;
    const int64_t row0 = int64_t(blockIdx.x / kCl) * kGemmM, gr = row0 + r;
    const bool valid = gr < a.n;
    const int nst = a.mode == kFusedValueGrad ? 9 : 5;
    // gradient outputs of this rank: grad-head columns j = k + 1 and back-propagated
    // columns k, both within [rank kOut, (rank + 1) kOut)
    const int k_lo = max(0, int(rank) * kOut - 1), k_hi = min(kMlpIn, int(rank) * kOut + kOut);
    // this rank's columns of a 256-wide tile start at byte own_off of each A tile
    const uint32_t own_off = rank * Cfg::kRankBytes;

    auto sB = [&](int st) { return sB0 + uint32_t(kBB > 1 ? (st & 1) : 0) * Cfg::kSmemB; };
    auto bar_load = [&](int st) { return bar_load0 + uint32_t(kBB > 1 ? (st & 1) : 0) * 8u; };
    auto issue_load = [&](int st) {
        const FusedStage fs = c_fstage[st];
        const int atoms = fs.K / 64;
        const int nc = fs.N / kCl;
        const uint32_t bar = bar_load(st);
        mbar_expect_tx(bar, uint32_t(atoms) * uint32_t(nc) * 128u);
        for (int at = 0; at < atoms; ++at)
            tma_load_2d(sB(st) + uint32_t(at) * uint32_t(nc) * 128u, fused_map(maps, fs.map), at * 64,
                        int(rank) * nc, bar);
    };
    // thread 0's record of what is in flight, drained (bounded) before exit
    int loads_out = 0, loads_done = 0;

    if (tid == 0) {
        mbar_init(bar_load0, 1);
        mbar_init(bar_load0 + 8u, 1);
        mbar_init(bar_mma, 1);
        mbar_init(bar_a0, 1);
        mbar_init(bar_a0 + 8u, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(Cfg::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    if (kCl > 1) cluster_barrier();       // every rank has started and initialised its barriers
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (tid == 0) {
        issue_load(0);
        ++loads_out;
        if (kBB > 1 && nst > 1) {
            issue_load(1);
            ++loads_out;
        }
    }

    // The prologue stages the slab's input rows and H in a part of the activation
    // tiles that stage 0 does not read (atoms 1..3 of the single tile, or the
    // second tile), with row strides of 49 floats so that column reads across a
    // warp hit distinct banks.
    constexpr int kLd = kMlpIn + 2;
    float* u_s = reinterpret_cast<float*>(smem_raw + (base - raw) +
                                          (Cfg::kABufs > 1 ? kFSmemA : kFAtomA));   // [128][49]
    float* h_s = u_s + kGemmM * kLd;                                                  // [47][49]
    constexpr int kNt = Cfg::kThreads;
    {
        // every load of the prologue is issued before any store, so that their
        // latencies overlap (coalesced: the slab's rows are contiguous in memory)
        constexpr int kNu = (kGemmM * kMlpIn + kNt - 1) / kNt;
        constexpr int kNh = (kMlpIn * kMlpIn + kNt - 1) / kNt;
        constexpr int kNb = (kFBiasFloats + kNt - 1) / kNt;
        float uv[kNu], hv[kNh], bv[kNb];
        float wv = 0.0f;
#pragma unroll
        for (int i = 0; i < kNu; ++i) {
            const int e = tid + i * kNt, rr = e / kMlpIn;
            uv[i] = (e < kGemmM * kMlpIn && row0 + rr < a.n) ? fused_in(a, row0 + rr, e - rr * kMlpIn) : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < kNh; ++i) {
            const int e = tid + i * kNt;
            hv[i] = (a.Hq && e < kMlpIn * kMlpIn) ? a.Hq[e] : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < kNb; ++i) {
            const int e = tid + i * kNt;
            const int l = e < 4 * kMlpHidden ? e / kMlpHidden : 4;
            bv[i] = e < kFBiasFloats ? a.bias[l][e - l * kMlpHidden] : 0.0f;
        }
        if (tid < kMlpHidden) wv = __bfloat162float(a.w4[tid]);
#pragma unroll
        for (int i = 0; i < kNu; ++i) {
            const int e = tid + i * kNt, rr = e / kMlpIn;
            if (e < kGemmM * kMlpIn) u_s[rr * kLd + (e - rr * kMlpIn)] = uv[i];
        }
#pragma unroll
        for (int i = 0; i < kNh; ++i) {
            const int e = tid + i * kNt;
            if (e < kMlpIn * kMlpIn) h_s[(e / kMlpIn) * kLd + e % kMlpIn] = hv[i];
        }
#pragma unroll
        for (int i = 0; i < kNb; ++i) {
            const int e = tid + i * kNt;
            if (e < kFBiasFloats) bias_s[e] = bv[i];
        }
        if (tid < kMlpHidden) w4_s[tid] = wv;
    }
    __syncthreads();
    if (grp == 0) {
        // the standardized input row: (theta - mean) / std for k < 47, zero
        // padding (every rank builds the whole tile, locally)
        float d[16];
#pragma unroll
        for (int c0 = 0; c0 < kMlpInPad; c0 += 16) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int k = c0 + j;
                d[j] = (valid && k < kMlpIn) ? (u_s[r * kLd + k] - a.xm[k]) / a.xs[k] : 0.0f;
            }
            store_act16(base, r, c0, d);
            if (a.tr_act && valid && rank == 0) trace_row<true>(a.tr_act + gr * kMlpHidden + c0, 16, d);
        }
    }
    if (a.Hq) {
        // quadratic baseline: gbase = -(H u)_k for this rank's gradient outputs,
        // one (row, k) dot product per thread in turn, each sum in the order j = 0..46
        // (warp group 0 builds the input tile meanwhile)
        // Four k per task share each u_j load (four independent sums).
        const int nk = k_hi - k_lo, ng = (nk + 3) / 4;
        for (int e = tid - 128; grp > 0 && e < kGemmM * ng; e += kNt - 128) {
            const int rr = e / ng, k0 = k_lo + 4 * (e - rr * ng);
            const float* uu = u_s + rr * kLd;
            float hu[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int j = 0; j < kMlpIn; ++j) {
                const float uj = uu[j];
#pragma unroll
                for (int t = 0; t < 4; ++t) hu[t] = fmaf(h_s[min(k0 + t, kMlpIn - 1) * kLd + j], uj, hu[t]);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (k0 + t < k_hi) gbase_s[rr * Cfg::kGb + (k0 + t - k_lo)] = -hu[t];
        }
        __syncthreads();
        if (tid < kGemmM && valid) {
            // the rank's share of u^T H u, in the order k = rank kOut ..
            float qd = 0.0f;
            for (int k = max(k_lo, int(rank) * kOut); k < k_hi; ++k)
                qd = fmaf(u_s[r * kLd + k], -gbase_s[r * Cfg::kGb + (k - k_lo)], qd);
            const uint32_t qa = smem_u32(qpart_s + rank * kGemmM + r);
            if (kCl > 1) {
                asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(map_rank(qa, 0u)), "f"(qd) : "memory");
            } else {
                qpart_s[r] = qd;
            }
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (kCl > 1) cluster_barrier();       // the baseline shares have reached rank 0
    tc_fence_after();

    const uint32_t tlane = tmem + (uint32_t(32 * q) << 16);
    const bool need_g = a.mode == kFusedValueGrad;          // gelu'(z) for the back-propagation
    constexpr int kGc = Cfg::kGc;
    for (int st = 0; st < nst; ++st) {
        const FusedStage fs = c_fstage[st];
        const int nc = fs.N / kCl;                       // this rank's columns of the stage
        const int cg0 = int(rank) * nc;                  // the first of them
        const int cbeg = grp * kGc;                      // this warp group's first local column
        const uint32_t curA = base + uint32_t(Cfg::kABufs > 1 ? (st & 1) : 0) * kFSmemA;
        const uint32_t nxtA = base + uint32_t(Cfg::kABufs > 1 ? ((st + 1) & 1) : 0) * kFSmemA;
        const uint32_t nxtBar = bar_a0 + uint32_t((st + 1) & 1) * 8u;   // the peers' barrier of that tile
        // the seed (stage 4) and the backward stages cover this rank's 256 / kCl columns
        const int hbeg = int(rank) * (kMlpHidden / kCl) + cbeg;
        // the hidden layer whose gelu'(z) this stage needs; from global scratch the
        // first 16 are requested before the MMA completes
        int glayer = -1;
        if (st == 4 && need_g) glayer = 3;
        else if (st >= 5 && st < 8) glayer = 7 - st;
        const float* gsrc = (glayer >= 0 && !Cfg::kGInTmem) ? a.gscr[glayer] + gr * kMlpHidden : nullptr;
        float4 gnext[4];
        if (gsrc && s_ok) load_g16(gsrc + hbeg, gnext);
        if (tid == 0) {
            bool ok = s_ok != 0;
            if (kBB > 1 && st >= 1 && st + 1 < nst && ok) {
                issue_load(st + 1);              // into the buffer MMA(st - 1) has finished with
                ++loads_out;
            }
            if (kCl > 1 && st >= 1) {
                // the peers' columns of this stage's tile (sent after their epilogues)
                const uint32_t bar = bar_a0 + uint32_t(st & 1) * 8u;
                const uint32_t par = uint32_t(((st - 1) >> 1) & 1);
                mbar_expect_tx(bar, uint32_t(kCl - 1) * Cfg::kRankBytes);
                if (!mbar_wait(bar, par, ok ? a.err : nullptr, 5)) ok = false;
            }
            const uint32_t ph = uint32_t(kBB > 1 ? ((st >> 1) & 1) : (st & 1));
            if (ok) {
                ok = mbar_wait(bar_load(st), ph, a.err, 3);
                if (ok) ++loads_done;
            }
            if (ok) {
                tc_fence_after();
                const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t(nc) >> 3) << 17) |
                                       ((uint32_t(kGemmM) >> 4) << 24);
                for (int k = 0; k < fs.K / 16; ++k) {
                    const uint32_t at = uint32_t(k >> 2), kk = uint32_t(k & 3);
                    const uint64_t da = smem_desc(curA + at * kFAtomA + kk * 32u);
                    const uint64_t db = smem_desc(sB(st) + at * uint32_t(nc) * 128u + kk * 32u);
                    tc_mma(tmem, da, db, idesc, k > 0 ? 1u : 0u);
                }
                tc_commit(bar_mma);
                ok = mbar_wait(bar_mma, uint32_t(st & 1), a.err, 4);
                if (!ok) mbar_wait(bar_mma, uint32_t(st & 1), nullptr, 0);   // MMAs in flight (bounded)
                else if (kBB == 1 && st + 1 < nst) {
                    issue_load(st + 1);
                    ++loads_out;
                }
            }
            s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        tc_fence_after();
        if (s_ok) {
            if (st < 4) {
                // hidden layer: z = acc + b; h = gelu(z) into this rank's columns of
                // the next tile; gelu'(z) (back-propagation only) to TMEM or scratch
                const float* bias = bias_s + st * kMlpHidden;
                float* gs = a.gscr[st] + gr * kMlpHidden;
#pragma unroll 1
                for (int c0 = cbeg; c0 < cbeg + kGc; c0 += 16) {
                    const int cg = int(rank) * (kMlpHidden / kCl) + c0;
                    float v[16], g[16];
                    tmem_ld16(tlane + uint32_t(c0), v);
                    if (a.tr_acc && valid)
                        trace_row<false>(a.tr_acc + st * a.tr_stride + gr * kMlpHidden + cg, 16, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float z = v[j] + bias[cg + j];
                        const float e = erf_gelu(z);
                        v[j] = gelu_e(z, e);
                        if (need_g) g[j] = gelu_grad_e(z, e);
                    }
                    if (need_g) {
                        if (Cfg::kGInTmem) {
                            tmem_st16(tlane + uint32_t(64 + 64 * st + c0), g);
                        } else {
                            float4* g4 = reinterpret_cast<float4*>(gs + cg);
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                g4[i] = make_float4(g[4 * i], g[4 * i + 1], g[4 * i + 2], g[4 * i + 3]);
                        }
                    }
                    store_act16(nxtA, r, cg, v);
                    if (a.tr_act && valid)
                        trace_row<true>(a.tr_act + (st + 1) * a.tr_stride + gr * kMlpHidden + cg, 16, v);
                }
            } else if (st == 4) {
                // output layer: y = acc + b_4 for this rank's columns j = cg0 ..
                const float* b4 = bias_s + 4 * kMlpHidden;
                if (grp == 0 && (a.mode == kFusedGradHead || rank == 0 || a.tr_acc)) {
                    float v[48];
                    tmem_ld_cols<kOutLd>(tlane, v);
                    if (a.tr_acc && valid) {
#pragma unroll
                        for (int j = 0; j < kOutLd; ++j)
                            if (cg0 + j < kMlpOut) a.tr_acc[4 * a.tr_stride + gr * kMlpHidden + cg0 + j] = v[j];
                    }
                    if (valid && rank == 0) {
                        const float y0 = v[0] + b4[0];
                        y0_s[r] = y0;
                        float base_r = 0.0f;
                        if (a.Hq) {
                            float qsum = 0.0f;
                            for (int c = 0; c < kCl; ++c) qsum += qpart_s[c * kGemmM + r];
                            base_r = -0.5f * qsum;
                        }
                        fused_out_ll(a, gr, y0 * a.ys + a.ym + base_r);
                    }
                    if (valid && a.mode == kFusedGradHead) {
                        // output j = 1 + k is d ll / d x_k
#pragma unroll
                        for (int jj = 0; jj < kOutLd; ++jj) {
                            const int j = cg0 + jj;
                            if (j < 1 || j >= kMlpOut) continue;
                            const int k = j - 1;
                            const float yk = v[jj] + b4[j];
                            fused_out_grad(a, gr, k, yk * a.ys / a.xs[k] +
                                                         (a.Hq ? gbase_s[r * Cfg::kGb + (k - k_lo)] : 0.0f));
                        }
                    }
                }
                if (need_g) {
                    // seed: dz_4 = (one-hot of the value output) W_4 * gelu'(z_4), for
                    // this rank's columns of the 256-wide tile
#pragma unroll 1
                    for (int c = 0; c < kGc; c += 16) {
                        const int c0 = hbeg + c;
                        float gg[16];
                        if (Cfg::kGInTmem) {
                            tmem_ld16(tlane + uint32_t(64 + 64 * 3 + cbeg + c), gg);
                        } else {
                            const float* gn = reinterpret_cast<const float*>(gnext);
#pragma unroll
                            for (int j = 0; j < 16; ++j) gg[j] = gn[j];
                            if (c + 16 < kGc) load_g16(gsrc + c0 + 16, gnext);
                        }
                        float d[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) d[j] = (valid ? w4_s[c0 + j] : 0.0f) * gg[j];
                        store_act16(nxtA, r, c0, d);
                        if (a.tr_act && valid)
                            trace_row<true>(a.tr_act + 5 * a.tr_stride + gr * kMlpHidden + c0, 16, d);
                    }
                }
            } else if (st < 8) {
                // back through layer 8 - st: dz = acc * gelu'(z)
#pragma unroll 1
                for (int c = 0; c < kGc; c += 16) {
                    const int c0 = cbeg + c, cg = hbeg + c;
                    float gg[16];
                    if (Cfg::kGInTmem) {
                        tmem_ld16(tlane + uint32_t(64 + 64 * glayer + c0), gg);
                    } else {
                        const float* gn = reinterpret_cast<const float*>(gnext);
#pragma unroll
                        for (int j = 0; j < 16; ++j) gg[j] = gn[j];
                        if (c + 16 < kGc) load_g16(gsrc + cg + 16, gnext);
                    }
                    float v[16];
                    tmem_ld16(tlane + uint32_t(c0), v);
                    if (a.tr_acc && valid)
                        trace_row<false>(a.tr_acc + st * a.tr_stride + gr * kMlpHidden + cg, 16, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = v[j] * gg[j];
                    store_act16(nxtA, r, cg, v);
                    if (a.tr_act && valid)
                        trace_row<true>(a.tr_act + (st + 1) * a.tr_stride + gr * kMlpHidden + cg, 16, v);
                }
            } else if (grp == 0) {
                // dx = dz_1 W_0: the gradient of the value output in the standardized
                // inputs, this rank's columns k = cg0 ..
                float v[48];
                tmem_ld_cols<kOutLd>(tlane, v);
                if (a.tr_acc && valid) {
#pragma unroll
                    for (int j = 0; j < kOutLd; ++j)
                        if (cg0 + j < kMlpIn) a.tr_acc[8 * a.tr_stride + gr * kMlpHidden + cg0 + j] = v[j];
                }
                if (valid) {
#pragma unroll
                    for (int jj = 0; jj < kOutLd; ++jj) {
                        const int k = cg0 + jj;
                        if (k >= kMlpIn) continue;
                        fused_out_grad(a, gr, k, v[jj] * a.ys / a.xs[k] +
                                                     (a.Hq ? gbase_s[r * Cfg::kGb + (k - k_lo)] : 0.0f));
                    }
                }
            }
        }
        fence_async_smem();                  // this CTA's tile writes, before the async proxy reads them
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // send this rank's columns of the next tile to every other rank (even after a
        // failure, so that no rank waits for them in vain)
        if (kCl > 1 && st + 1 < nst) {
            if (tid == 0) {
#pragma unroll
                for (int d = 1; d < kCl; ++d)
                    bulk_copy_to_rank(nxtA + own_off, Cfg::kRankBytes, nxtBar, (rank + uint32_t(d)) % kCl);
            }
        }
    }
    // drain (bounded) what thread 0 left in flight after a failure: weight
    // copies it issued but did not wait for, and the peers' tile copies
    if (tid == 0) {
        for (int i = loads_done; i < loads_out; ++i) {
            const int st = i;             // loads are issued and waited in stage order
            mbar_wait(bar_load(st), uint32_t(kBB > 1 ? ((st >> 1) & 1) : (st & 1)), nullptr, 0);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (kCl > 1) cluster_barrier();       // no rank exits while a copy into it may be in flight
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(Cfg::kTmemCols)
                     : "memory");
    }
}

template <int kCl>
cudaError_t configure_fused(int dev) {
    static bool configured[64] = {};
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        cudaError_t ce = cudaFuncSetAttribute(k_mlp_fused<kCl>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              int(FusedCfg<kCl>::kSmem));
        if (ce != cudaSuccess) return ce;
        configured[dev] = true;
    }
    return cudaSuccess;
}

template <int kCl>
cudaLaunchConfig_t fused_config(unsigned grid, cudaStream_t s, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(FusedCfg<kCl>::kThreads);
    cfg.dynamicSmemBytes = FusedCfg<kCl>::kSmem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// How many clusters of kCl fused CTAs the device runs at once (0 if unknown).
template <int kCl>
int fused_max_clusters(int dev) {
    static int cached[64] = {};
    if (dev < 0 || dev >= 64) return 0;
    if (!cached[dev]) {
        if (configure_fused<kCl>(dev) != cudaSuccess) return 0;
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = fused_config<kCl>(unsigned(kCl), nullptr, attr);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_mlp_fused<kCl>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        cached[dev] = n > 0 ? n : -1;
    }
    return cached[dev] > 0 ? cached[dev] : 0;
}

template <int kCl>
cudaError_t launch_fused_cl(const MlpFusedMaps& maps, const MlpFusedArgs& a, cudaStream_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t ce = configure_fused<kCl>(dev);
    if (ce != cudaSuccess) return ce;
    const unsigned grid = unsigned((a.n + kGemmM - 1) / kGemmM) * kCl;
    if (kCl == 1) {
        k_mlp_fused<1><<<grid, FusedCfg<1>::kThreads, FusedCfg<1>::kSmem, s>>>(maps, a);
        return cudaGetLastError();
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = fused_config<kCl>(grid, s, attr);
    return cudaLaunchKernelEx(&cfg, k_mlp_fused<kCl>, maps, a);
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


// The widest cluster whose clusters all run at once for n rows (one 128-row
// slab per cluster); 1 when even two-CTA clusters would need a second wave.
int fused_cluster_size(int64_t n) {
    int dev = 0;
    cudaGetDevice(&dev);
    const int64_t slabs = (n + kGemmM - 1) / kGemmM;
    if (slabs <= fused_max_clusters<4>(dev)) return 4;
    if (slabs <= fused_max_clusters<2>(dev)) return 2;
    return 1;
}

cudaError_t launch_mlp_fused(const MlpFusedMaps* maps, const MlpFusedArgs& a, cudaStream_t s, int cl) {
    const bool f64 = a.z64 != nullptr;
    if (a.n <= 0 || a.mode < kFusedValue || a.mode > kFusedGradHead ||
        (f64 ? (!a.zc || !a.ll64 || (a.mode != kFusedValue && !a.g64))
             : (!a.theta || !a.loglik || (a.mode != kFusedValue && !a.grad))))
        return cudaErrorInvalidValue;
    if (cl == 0) cl = fused_cluster_size(a.n);
    switch (cl) {
        case 1: return launch_fused_cl<1>(maps[0], a, s);
        case 2: return launch_fused_cl<2>(maps[1], a, s);
        case 4: return launch_fused_cl<4>(maps[2], a, s);
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
