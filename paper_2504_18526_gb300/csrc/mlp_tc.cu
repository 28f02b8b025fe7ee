// Fused forward pass of the element-patch MLP on the fifth-generation tensor
// cores (tcgen05): one 128-row tile of patch rows per step of a persistent
// CTA, all three layers chained through tensor memory.
//
//   layer 1: the patch rows are gathered from the FP64 residual, scaled by
//            1/s and rounded to BF16 straight into the swizzled A panels in
//            shared memory (no patch matrix in global memory); W1^T is
//            resident in shared memory (loaded once per CTA by TMA);
//            tcgen05.mma accumulates X W1 in TMEM (FP32);
//   epilogue: TMEM -> registers (tcgen05.ld), + bias, tanh, BF16 -> the A
//            panels of the next layer;
//   layer 2 and 3 alike (W2^T, W3^T resident); the last epilogue adds the
//            bias and writes z = r + s y (FP64) to the output field.
//
// One thread issues the MMAs and TMA copies; every wait on an mbarrier is
// bounded (about 1 s) and records an error flag instead of hanging.  The
// CTA frees its TMEM before it returns, also after an error.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ds.cuh"
#include "mlp_tc.h"
#include "tc.cuh"

namespace sisdc {

namespace {

constexpr int TILE_M = 128;
constexpr int THREADS = 512;                     // 16 warps: 4 per TMEM lane quarter
constexpr uint32_t PANEL_A = TILE_M * 128;      // bytes of one 64-wide K panel of a 128-row tile
constexpr uint32_t TMEM_COLS = 128;

struct Layout {
    uint32_t w1, w2, w3, xs, hs, bias, nb, bars, total;
};

__host__ __device__ inline Layout layout(int nP1, int H, int N3) {
    Layout L{};
    uint32_t o = 0;
    L.w1 = o; o += (uint32_t)nP1 * H * 128;
    L.w2 = o; o += 2u * H * 128;
    L.w3 = o; o += 2u * N3 * 128;
    L.xs = o; o += 2 * PANEL_A;                  // double-buffered gather panels
    L.hs = o; o += 2 * PANEL_A;
    L.bias = o; o += (uint32_t)(2 * H + N3) * 4;
    L.nb = o; o += TILE_M * 10 * 4;              // per tile row: nine neighbour offsets, 1/s
    o = (o + 15) & ~15u;
    L.bars = o; o += 64;
    L.total = o;
    return L;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
    return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}

// Threads: 16 warps.  Warp w reads TMEM lane quarter w % 4 (rows 32 (w % 4) ..
// + 31) and takes the 16-column accumulator chunks c with c % 4 == w / 4 in
// the epilogues; all threads gather the patch panels.  Layer 1 runs over the
// K panels with two gather buffers: panel p is gathered into buffer p % 2
// while the MMAs of panel p - 1 run; a buffer is refilled only after the
// commit of the MMAs that read it has arrived on that buffer's barrier.
__global__ void __launch_bounds__(THREADS, 1) k_mlp_fwd_tc(const MlpTcArgs a, const __grid_constant__ CUtensorMap m1,
                                                           const __grid_constant__ CUtensorMap m2,
                                                           const __grid_constant__ CUtensorMap m3) {
    extern __shared__ uint8_t smraw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    const Layout L = layout(a.nP1, a.H, a.N3);
    uint8_t* W1s = base + L.w1;
    uint8_t* W2s = base + L.w2;
    uint8_t* W3s = base + L.w3;
    uint8_t* Xs = base + L.xs;
    uint8_t* Hs = base + L.hs;
    float* sb1 = reinterpret_cast<float*>(base + L.bias);
    float* sb2 = sb1 + a.H;
    float* sb3 = sb2 + a.H;
    int* snb = reinterpret_cast<int*>(base + L.nb);           // [row][9] field offsets (int: NV < 2^31)
    float* ssi = reinterpret_cast<float*>(snb + TILE_M * 9);   // [row] 1/s
    uint64_t* tma_bar = reinterpret_cast<uint64_t*>(base + L.bars);
    uint64_t* mma_bar = tma_bar + 1;
    uint64_t* xbar = tma_bar + 2;                // [2]: MMAs that read gather buffer b are done
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tma_bar + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, cgrp = warp >> 2;
    for (int t = tid; t < a.H; t += blockDim.x) {
        sb1[t] = a.b1[t];
        sb2[t] = a.b2[t];
    }
    for (int t = tid; t < a.N3; t += blockDim.x) sb3[t] = t < a.q ? a.b3[t] : 0.f;
    if (tid == 0) {
        tc::mbar_init(tma_bar, 1);
        tc::mbar_init(mma_bar, 1);
        tc::mbar_init(xbar, 1);
        tc::mbar_init(xbar + 1, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    // resident weights: W1^T (nP1 panels), W2^T and W3^T (two panels each)
    if (tid == 0) {
        const uint32_t bytes = (uint32_t)(a.nP1 + 2) * a.H * 128 + 2u * a.N3 * 128;
        tc::mbar_arrive_expect_tx(tma_bar, bytes);
        for (int p = 0; p < a.nP1; ++p) tc::tma_load_2d(W1s + (size_t)p * a.H * 128, &m1, tma_bar, 64 * p, 0);
        for (int p = 0; p < 2; ++p) {
            tc::tma_load_2d(W2s + (size_t)p * a.H * 128, &m2, tma_bar, 64 * p, 0);
            tc::tma_load_2d(W3s + (size_t)p * a.N3 * 128, &m3, tma_bar, 64 * p, 0);
        }
    }
    bool ok = __syncthreads_and(tc::mbar_wait(tma_bar, 0)) != 0;
    uint32_t mph = 0;
    uint32_t xcommit[2] = {0, 0}, xwait[2] = {0, 0};   // commits to / waits consumed on xbar[b]
    const uint32_t id12 = tc::idesc_bf16_f32(TILE_M, a.H);
    const uint32_t id3 = tc::idesc_bf16_f32(TILE_M, a.N3);
    const int k1 = (a.n_in + 15) / 16, kh = a.H / 16;           // MMA K steps of 16
    const int nel = a.nex * a.ney;
    const long long ntiles = (a.rows + TILE_M - 1) / TILE_M;
    const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16);
    const int row_e = quarter * 32 + lane;                      // the epilogue row of this thread

    // epilogue of layers 1 and 2: tanh(acc + bias) in BF16 into the A panels Hs
    auto hidden_epilogue = [&](const float* bias) {
        for (int c0 = 16 * cgrp; c0 < a.H; c0 += 64) {
            float v[16];
            tc::tmem_ld16(tq + (uint32_t)c0, v);
            uint32_t w[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) w[k] = pack_bf16(tanhf(v[2 * k] + bias[c0 + 2 * k]), tanhf(v[2 * k + 1] + bias[c0 + 2 * k + 1]));
            uint8_t* panel = Hs + (c0 >> 6) * PANEL_A;
            const int k0 = c0 & 63;
            *reinterpret_cast<uint4*>(panel + tc::sw128_offset(row_e, k0)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4*>(panel + tc::sw128_offset(row_e, k0 + 8)) = make_uint4(w[4], w[5], w[6], w[7]);
        }
    };
    auto issue = [&](const uint8_t* Bbase, uint32_t bpanel, int ksteps, uint32_t idesc) {
        for (int k = 0; k < ksteps; ++k) {
            const int p = k >> 2, s4 = k & 3;
            const uint64_t ad = tc::sdesc_k_sw128(tc::smem_u32(Hs + p * PANEL_A + s4 * 32));
            const uint64_t bd = tc::sdesc_k_sw128(tc::smem_u32(Bbase + p * bpanel + s4 * 32));
            tc::mma_bf16(tmem, ad, bd, idesc, k == 0 ? 0u : 1u);
        }
        tc::mma_commit(mma_bar);
    };
    // every thread waits; ok stays uniform over the block
    auto wait_mma = [&]() {
        const bool w = tc::mbar_wait(mma_bar, mph);
        mph ^= 1;
        ok = __syncthreads_and(w && ok) != 0;
        tc::fence_after_sync();
    };
    // consume the outstanding commit on gather buffer b (at most one)
    auto drain = [&](int b) {
        bool w = true;
        if (xwait[b] < xcommit[b]) {
            w = tc::mbar_wait(xbar + b, xwait[b] & 1);
            ++xwait[b];
        }
        return w;
    };

    // the gather: a thread always fills 16-byte chunk kc = tid % 8 of a panel
    // row, for rows tid / 8 and tid / 8 + 64 of the tile
    constexpr int RPT = TILE_M * 8 / THREADS;                   // rows per thread (2)
    const int kc = tid & 7, rbase = tid >> 3;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long row0 = tile * TILE_M;
        // per row: the nine neighbour elements' offsets into the field, and 1/s
        // (the first barrier of the panel loop publishes them)
        for (int t = tid; t < TILE_M * 9; t += THREADS) {
            const int r = t / 9, k = t - r * 9;
            const long long grow = row0 + r;
            int off = 0;
            if (grow < a.rows) {
                const int comp = (int)(grow / nel), el = (int)(grow - (long long)comp * nel);
                const int ex = el % a.nex, ey = el / a.nex;
                const int dy = k / 3 - 1, dx = k % 3 - 1;
                const int en = ((ey + dy + a.ney) % a.ney) * a.nex + (ex + dx + a.nex) % a.nex;
                off = (comp * nel + en) * a.q;
            }
            snb[t] = off;
            if (k == 0) ssi[r] = grow < a.rows ? a.sinv[grow] : 0.f;
        }
        // ---- layer 1: panels of the gathered patch rows ----------------------------
        for (int p = 0; p < a.nP1 && ok; ++p) {
            const int b = p & 1;
            uint8_t* Xb = Xs + b * PANEL_A;
            // this thread's eight input columns of panel p: (neighbour, node), or
            // the feature (nb = 9), or padding (nb = 10)
            int nbk[8], nodek[8];
            {
                const int t0 = 64 * p + 8 * kc;
                int nb = t0 / a.q, node = t0 - nb * a.q;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int t = t0 + e;
                    nbk[e] = t < 9 * a.q ? nb : (t == 9 * a.q ? 9 : 10);
                    nodek[e] = node;
                    if (++node == a.q) {
                        node = 0;
                        ++nb;
                    }
                }
            }
            ok = __syncthreads_and(drain(b) && ok) != 0;      // the MMAs that read Xb are done
            if (!ok) break;
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const int r = rbase + 64 * i;
                const bool in = row0 + r < a.rows;
                const int* nb9 = snb + r * 9;
                const float si = ssi[r];
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int nb = nbk[e];
                    float x = 0.f;
                    if (in && nb < 9) x = d2f_int(__ldg(a.field + nb9[nb] + nodek[e])) * si;
                    else if (in && nb == 9) x = a.feat;
                    v[e] = x;
                }
                *reinterpret_cast<uint4*>(Xb + tc::sw128_offset(r, 8 * kc)) =
                    make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
            }
            tc::fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                const int ks = min(4, k1 - 4 * p);
                for (int kk = 0; kk < ks; ++kk) {
                    const uint64_t ad = tc::sdesc_k_sw128(tc::smem_u32(Xb + kk * 32));
                    const uint64_t bd = tc::sdesc_k_sw128(tc::smem_u32(W1s + (size_t)p * a.H * 128 + kk * 32));
                    tc::mma_bf16(tmem, ad, bd, id12, (p == 0 && kk == 0) ? 0u : 1u);
                }
                tc::mma_commit(xbar + b);
            }
            ++xcommit[b];
        }
        // all layer-1 MMAs complete (the last commits of both buffers)
        ok = __syncthreads_and(drain(0) && drain(1) && ok) != 0;
        tc::fence_after_sync();
        if (!ok) break;
        // ---- layer 2 ---------------------------------------------------------
        hidden_epilogue(sb1);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue(W2s, (uint32_t)a.H * 128, kh, id12);
        }
        wait_mma();
        if (!ok) break;
        // ---- layer 3 ---------------------------------------------------------
        hidden_epilogue(sb2);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue(W3s, (uint32_t)a.N3 * 128, kh, id3);
        }
        wait_mma();
        if (!ok) break;
        // ---- output: z (+)= r + s (acc + b3) ---------------------------------
        {
            const long long grow = row0 + row_e;
            const float s = grow < a.rows ? a.s[grow] : 0.f;
            for (int c0 = 16 * cgrp; c0 < a.N3; c0 += 64) {
                float v[16];
                tc::tmem_ld16(tq + (uint32_t)c0, v);
                if (grow < a.rows)
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int col = c0 + k;
                        if (col < a.q) {
                            const long long o = grow * a.q + col;
                            const double val = a.field[o] + f2d_int((v[k] + sb3[col]) * s);
                            a.z[o] = a.add ? a.z[o] + val : val;
                        }
                    }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicOr(a.err, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

bool mlp_tc_eligible(int n_in, int H, int q, size_t* smem) {
    if (H < 16 || H > 128 || H % 16 != 0 || q < 1 || q > 128 || n_in < 1) return false;
    const int nP1 = (n_in + 63) / 64;
    const int N3 = (q + 15) / 16 * 16;
    const Layout L = layout(nP1, H, N3);
    const size_t need = (size_t)L.total + 1024;
    if (smem) *smem = need;
    return need <= 227 * 1024;
}

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}
}  // namespace

// [rows][cols] BF16 row-major (cols a multiple of 64), boxes of 64 x box_rows,
// 128-byte swizzle
bool mlp_tc_encode(void* map, const void* ptr, int rows, int cols, int box_rows) {
    EncodeTiledFn fn = encoder();
    if (!fn || cols % 64 != 0 || box_rows < 1 || box_rows > 256) return false;
    if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1u, 1u};
    return fn(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims,
              strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t mlp_tc_forward(const MlpTcArgs& a, const void* m1, const void* m2, const void* m3, int nsm,
                           cudaStream_t s) {
    size_t smem = 0;
    if (!mlp_tc_eligible(a.n_in, a.H, a.q, &smem)) return cudaErrorInvalidValue;
    if (a.nP1 != (a.n_in + 63) / 64 || a.N3 != (a.q + 15) / 16 * 16) return cudaErrorInvalidValue;
    if (a.rows * (long long)a.q >= (1LL << 31)) return cudaErrorInvalidValue;   // int field offsets
    cudaError_t e = cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long ntiles = (a.rows + TILE_M - 1) / TILE_M;
    const int grid = (int)(ntiles < nsm ? ntiles : nsm);
    k_mlp_fwd_tc<<<grid, THREADS, smem, s>>>(a, *reinterpret_cast<const CUtensorMap*>(m1),
                                         *reinterpret_cast<const CUtensorMap*>(m2),
                                         *reinterpret_cast<const CUtensorMap*>(m3));
    return cudaGetLastError();
}

// W1^T [H][K1p], W2^T [H][128], W3^T [N3][128] in BF16 from the FP32 master
// weights W1 [n_in][H], W2 [H][H], W3 [H][q] (zero padding)
__global__ void k_mlp_pack_tc(const float* __restrict__ W1, const float* __restrict__ W2, const float* __restrict__ W3,
                              int n_in, int H, int q, int K1p, int N3, __nv_bfloat16* __restrict__ W1T,
                              __nv_bfloat16* __restrict__ W2T, __nv_bfloat16* __restrict__ W3T) {
    const long long n1 = (long long)H * K1p, n2 = (long long)H * 128, n3 = (long long)N3 * 128;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n1 + n2 + n3;
         t += (long long)gridDim.x * blockDim.x) {
        if (t < n1) {
            const int h = (int)(t / K1p), k = (int)(t % K1p);
            W1T[t] = __float2bfloat16(k < n_in ? W1[(long long)k * H + h] : 0.f);
        } else if (t < n1 + n2) {
            const long long u = t - n1;
            const int h = (int)(u / 128), k = (int)(u % 128);
            W2T[u] = __float2bfloat16(k < H ? W2[(long long)k * H + h] : 0.f);
        } else {
            const long long u = t - n1 - n2;
            const int n = (int)(u / 128), k = (int)(u % 128);
            W3T[u] = __float2bfloat16(n < q && k < H ? W3[(long long)k * q + n] : 0.f);
        }
    }
}

cudaError_t mlp_tc_pack(const float* W1, const float* W2, const float* W3, int n_in, int H, int q, int K1p, int N3,
                        void* W1T, void* W2T, void* W3T, cudaStream_t s) {
    k_mlp_pack_tc<<<256, 256, 0, s>>>(W1, W2, W3, n_in, H, q, K1p, N3, static_cast<__nv_bfloat16*>(W1T),
                                      static_cast<__nv_bfloat16*>(W2T), static_cast<__nv_bfloat16*>(W3T));
    return cudaGetLastError();
}

}  // namespace sisdc
