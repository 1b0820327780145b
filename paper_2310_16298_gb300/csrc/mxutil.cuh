// Helpers shared by the matrixized kernels (2D and 3D).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <mutex>
#include <array>
#include <vector>

#include "plan.h"

#include "../../include/stencil.h"
#include "ptx.cuh"

namespace stx {
namespace mxu {

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

// Bounded mbarrier wait that also gives up once another role has failed.
// Between polls the warp sleeps briefly, so that waiting warps leave the
// issue slots (and the shared-memory pipe) to the warps doing the work.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    const long long t0 = clock64();
    while (!ptx::mbar_try_wait(bar, parity)) {
        __nanosleep(64);
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// TF32 high part by integer rounding (nearest, ties away from zero): the low
// 13 mantissa bits are cleared after adding half of their weight.
__device__ __forceinline__ uint32_t tf32_hi_bits(float x) {
    return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

// BF16 bits (upper half of the FP32 pattern) of x rounded to nearest, ties to
// even; finite inputs.
__device__ __forceinline__ uint32_t bf16_rn_bits(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}


// Operand formats of the matrixized kernels.  Both use, per MMA K-step, 8
// tensor-memory columns of A and two 16-byte chunks of B:
//   TF32 (kind::tf32): one element per column, K = 8 per MMA, parts hi/lo;
//   BF16 (kind::f16):  two elements per column, K = 16 per MMA, parts 0/1/2.
template <bool BF>
struct OpFmt {
    static constexpr int kKStep = BF ? 16 : 8;          // K per MMA
    static constexpr int kGroup = BF ? 16 : 8;          // input columns per tcgen05.st x8
    static constexpr uint32_t kFmt = BF ? 1u : 2u;      // instruction-descriptor A/B format
    static constexpr int kMaxParts = BF ? 3 : 2;
    __host__ __device__ static constexpr int window(int nb) {  // K window for nb outputs
        return ((nb + 8) + kKStep - 1) / kKStep * kKStep;
    }
    __host__ __device__ static constexpr int part_cols(int k) { return BF ? k / 2 : k; }
};

// Products per K step of a precision mode (see issue_products).
inline int products_for(int prec) {
    switch (prec) {
        case STENCIL_PREC_TF32X3: return 3;
        case STENCIL_PREC_BF16X2: return 3;
        case STENCIL_PREC_BF16X3: return 6;
        case STENCIL_PREC_BF16_W2: return 2;
    }
    return 1;
}

// Precisions the outer-product kernels run.
inline bool mx_precision(int prec) { return prec >= STENCIL_PREC_TF32 && prec <= STENCIL_PREC_BF16_W2; }

inline int operand_parts(int prec) {
    switch (prec) {
        case STENCIL_PREC_TF32X3: return 2;
        case STENCIL_PREC_BF16X2: return 2;
        case STENCIL_PREC_BF16X3: return 3;
    }
    return 1;
}

inline bool is_bf16(int prec) {
    return prec == STENCIL_PREC_BF16 || prec == STENCIL_PREC_BF16X2 || prec == STENCIL_PREC_BF16X3 ||
           prec == STENCIL_PREC_BF16_W2;
}

// Issue every K step of one product (A part PA, B part PB) into accumulator
// d; FIRST clears the accumulator with the first step.
template <bool BF, int KS, int PA, int PB, bool FIRST>
__device__ __forceinline__ void issue_product(uint32_t d, uint32_t a_base, int part_cols, uint64_t b_desc0,
                                              uint32_t bpart_bytes, int n, uint32_t idesc) {
    const uint32_t a = a_base + (uint32_t)(PA * part_cols);
    const uint64_t b = b_desc0 + (uint64_t)((PB * bpart_bytes) >> 4);
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
        const uint64_t bd = b + (uint64_t)((2 * ks * n * 16) >> 4);
        if (FIRST && ks == 0)
            ptx::mma_ts<BF, true>(d, a + 8 * ks, bd, idesc);
        else
            ptx::mma_ts<BF, false>(d, a + 8 * ks, bd, idesc);
    }
}

// Issue every product of one tile (A in tensor memory, B in shared memory)
// into accumulator d, smallest products first: nprod = 1 (x0*h0), 2 (x0*h1,
// x0*h0), 3 (x1*h0, x0*h1, x0*h0) or 6 (x0*h2, x1*h1, x2*h0, x1*h0, x0*h1,
// x0*h0).  Each product count is its own fixed sequence.
template <bool BF, int KS>
__device__ __forceinline__ void issue_products(uint32_t d, uint32_t a_base, int pc, uint64_t b0, uint32_t bpb,
                                               int n, uint32_t idesc, int nprod) {
    switch (nprod) {
        case 1:
            issue_product<BF, KS, 0, 0, true>(d, a_base, pc, b0, bpb, n, idesc);
            break;
        case 2:
            issue_product<BF, KS, 0, 1, true>(d, a_base, pc, b0, bpb, n, idesc);
            issue_product<BF, KS, 0, 0, false>(d, a_base, pc, b0, bpb, n, idesc);
            break;
        case 3:
            issue_product<BF, KS, 1, 0, true>(d, a_base, pc, b0, bpb, n, idesc);
            issue_product<BF, KS, 0, 1, false>(d, a_base, pc, b0, bpb, n, idesc);
            issue_product<BF, KS, 0, 0, false>(d, a_base, pc, b0, bpb, n, idesc);
            break;
        case 6:
            issue_product<BF, KS, 0, 2, true>(d, a_base, pc, b0, bpb, n, idesc);
            issue_product<BF, KS, 1, 1, false>(d, a_base, pc, b0, bpb, n, idesc);
            issue_product<BF, KS, 2, 0, false>(d, a_base, pc, b0, bpb, n, idesc);
            issue_product<BF, KS, 1, 0, false>(d, a_base, pc, b0, bpb, n, idesc);
            issue_product<BF, KS, 0, 1, false>(d, a_base, pc, b0, bpb, n, idesc);
            issue_product<BF, KS, 0, 0, false>(d, a_base, pc, b0, bpb, n, idesc);
            break;
    }
}

// Split kGroup input values into NP operand parts and write them to the
// warp's tensor-memory lanes at column c (part p at a_base + p*part_cols).
// The stores have completed when this returns.
template <bool BF, int NP>
__device__ __forceinline__ void split_store(const float* x, uint32_t a_base, int part_cols, int c) {
    if constexpr (!BF) {
        uint32_t h[8], l[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            h[e] = tf32_hi_bits(x[e]);
            if constexpr (NP > 1) l[e] = __float_as_uint(x[e] - __uint_as_float(h[e]));
        }
        if constexpr (NP > 1)
            ptx::tmem_st_x8_sync(a_base + (uint32_t)c, h, a_base + (uint32_t)(part_cols + c), l);
        else
            ptx::tmem_st_x8_sync(a_base + (uint32_t)c, h);
    } else {
        uint32_t w[NP][8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float r0a = x[2 * e], r0b = x[2 * e + 1];
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const uint32_t ba = bf16_rn_bits(r0a), bb = bf16_rn_bits(r0b);
                w[k][e] = ba | (bb << 16);
                if (k + 1 < NP) {
                    r0a -= __uint_as_float(ba << 16);
                    r0b -= __uint_as_float(bb << 16);
                }
            }
        }
        const uint32_t a0 = a_base + (uint32_t)(c / 2);
        if constexpr (NP == 1)
            ptx::tmem_st_x8_sync(a0, w[0]);
        else if constexpr (NP == 2)
            ptx::tmem_st_x8_sync(a0, w[0], a0 + (uint32_t)part_cols, w[1]);
        else
            ptx::tmem_st_x8_sync(a0, w[0], a0 + (uint32_t)part_cols, w[1], a0 + (uint32_t)(2 * part_cols), w[2]);
    }
}

// Split NGR groups of kGroup input values (x[g], written at column c0 + g *
// cstep) into NP operand parts each and write them all with one fused
// store-and-wait: the stores have completed when this returns.
template <bool BF, int NP, int NGR>
__device__ __forceinline__ void split_store_groups(const float (&x)[NGR][OpFmt<BF>::kGroup], uint32_t a_base,
                                                   int part_cols, int c0, int cstep) {
    uint32_t addr[NGR * NP];
    uint32_t w[NGR * NP][8];
#pragma unroll
    for (int g = 0; g < NGR; ++g) {
        const int c = c0 + cstep * g;
        if constexpr (!BF) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint32_t h = tf32_hi_bits(x[g][e]);
                w[g * NP][e] = h;
                if constexpr (NP > 1) w[g * NP + 1][e] = __float_as_uint(x[g][e] - __uint_as_float(h));
            }
#pragma unroll
            for (int k = 0; k < NP; ++k) addr[g * NP + k] = a_base + (uint32_t)(k * part_cols + c);
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                float r0a = x[g][2 * e], r0b = x[g][2 * e + 1];
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const uint32_t ba = bf16_rn_bits(r0a), bb = bf16_rn_bits(r0b);
                    w[g * NP + k][e] = ba | (bb << 16);
                    if (k + 1 < NP) {
                        r0a -= __uint_as_float(ba << 16);
                        r0b -= __uint_as_float(bb << 16);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < NP; ++k) addr[g * NP + k] = a_base + (uint32_t)(k * part_cols + c / 2);
        }
    }
    ptx::tmem_st_x8_sync_n<NGR * NP>(addr, w);
}

// Run-time part count (kernels not specialised on it).
template <bool BF>
__device__ __forceinline__ void split_store(const float* x, uint32_t a_base, int part_cols, int c, int nparts) {
    if (nparts == 1)
        split_store<BF, 1>(x, a_base, part_cols, c);
    else if (nparts == 2 || !BF)
        split_store<BF, 2>(x, a_base, part_cols, c);
    else
        split_store<BF, 3>(x, a_base, part_cols, c);
}

inline PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}


// Round to BF16 on the host (nearest, ties to even); finite inputs.
inline float bf16_round(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    u &= 0xFFFF0000u;
    float y;
    memcpy(&y, &u, 4);
    return y;
}

// Round to TF32 on the host (nearest, ties to even); finite inputs.
inline float tf32_round(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    u += 0xFFFu + ((u >> 13) & 1u);
    u &= ~0x1FFFu;
    float y;
    memcpy(&y, &u, 4);
    return y;
}


// Pack the banded operands of the given lines (line l: 2r+1 gather weights)
// as the MMA B operand, N = lines x nb rows, K-major 16-byte chunks:
// [part][k chunk][n = l*nb + q][16 bytes].  Row (n, k) holds the band entry
// H_l[k][q] = w_l[k - q - (4 - r)] (zero outside the band and for k >= nb + 8),
// split into TF32 hi/lo parts or three BF16 parts.  Returns the bytes of one
// part in *part_bytes.
// Banded operand of a block list: block j stacks, along K, the band of line
// blocks[j][0] (K rows 0 .. kh-1) over the band of line blocks[j][1] (rows
// kh .. 2kh-1); a null line contributes zeros.  Used when one TMEM lane holds
// two input rows side by side along K.
inline std::vector<unsigned char> pack_blocks(int r, const std::vector<std::array<const double*, 2>>& blocks, int nb,
                                              int kh, bool bf, uint32_t* part_bytes) {
    const int nblk = (int)blocks.size(), N = nblk * nb, kw = 2 * kh;
    const int epc = bf ? 8 : 4;  // elements per 16-byte chunk
    const int es = bf ? 2 : 4;
    const int parts = bf ? 3 : 2;
    const size_t pb = (size_t)(kw / epc) * N * 16;
    std::vector<unsigned char> out(parts * pb, 0);
    std::vector<double> band((size_t)(nb + 8) * nb);
    for (int j = 0; j < nblk; ++j)
        for (int e = 0; e < 2; ++e) {
            if (!blocks[j][e]) continue;
            band_operand(r, blocks[j][e], nb, 4, band.data());
            for (int kk = 0; kk < nb + 8; ++kk)
                for (int q = 0; q < nb; ++q) {
                    const int k = e * kh + kk;
                    float rem = (float)band[(size_t)kk * nb + q];
                    const size_t off = ((size_t)(k / epc) * N + (size_t)(j * nb + q)) * 16 + (size_t)(k % epc) * es;
                    for (int p = 0; p < parts; ++p) {
                        const float v = bf ? bf16_round(rem) : tf32_round(rem);
                        rem -= v;
                        if (bf) {
                            uint32_t u;
                            memcpy(&u, &v, 4);
                            const uint16_t h = (uint16_t)(u >> 16);
                            memcpy(&out[p * pb + off], &h, 2);
                        } else {
                            memcpy(&out[p * pb + off], &v, 4);
                        }
                    }
                }
        }
    *part_bytes = (uint32_t)pb;
    return out;
}

inline std::vector<unsigned char> pack_bands(int r, const std::vector<const double*>& lines, int nb, int kwin, bool bf,
                                             uint32_t* part_bytes) {
    const int L = (int)lines.size(), N = L * nb;
    const int epc = bf ? 8 : 4;  // elements per 16-byte chunk
    const int es = bf ? 2 : 4;
    const int parts = bf ? 3 : 2;
    const size_t pb = (size_t)(kwin / epc) * N * 16;
    std::vector<unsigned char> out(parts * pb, 0);
    std::vector<double> band((size_t)(nb + 8) * nb);
    for (int l = 0; l < L; ++l) {
        band_operand(r, lines[l], nb, 4, band.data());
        for (int k = 0; k < nb + 8; ++k)
            for (int q = 0; q < nb; ++q) {
                float rem = (float)band[(size_t)k * nb + q];
                const size_t off = ((size_t)(k / epc) * N + (size_t)(l * nb + q)) * 16 + (size_t)(k % epc) * es;
                for (int p = 0; p < parts; ++p) {
                    const float v = bf ? bf16_round(rem) : tf32_round(rem);
                    rem -= v;
                    if (bf) {
                        uint32_t u;
                        memcpy(&u, &v, 4);
                        const uint16_t h = (uint16_t)(u >> 16);
                        memcpy(&out[p * pb + off], &h, 2);
                    } else {
                        memcpy(&out[p * pb + off], &v, 4);
                    }
                }
            }
    }
    *part_bytes = (uint32_t)pb;
    return out;
}

}  // namespace mxu
}  // namespace stx
