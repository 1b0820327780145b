// Matrixized stencil sweep on the 5th-generation tensor cores (tcgen05).
//
// Scatter-mode formulation (Sec. 3): every coefficient line contributes, to
// an output block, the sum over its input vectors of (input vector) x
// (coefficient vector) outer products -- Eq. (final).  The kernels take the
// lines along the contiguous axis (the paper's orthogonal line orientation,
// Eq. (to-outer-product-2-star)), so for line a (input row offset a - r) and
// an output block of Nb columns
//
//     D[m, q] += sum_k A[m + a, k] * H_a[k, q],   H_a[k, q] = C^g[a, k - q - 4 + r]
//
// where A is the K = Nb + 8 column window of the input tile starting 4
// columns left of the block and H_a is the line's banded (Toeplitz) operand:
// the columns of H_a are the coefficient vectors of Eq. (co) / Eq. (final).
// One tcgen05.mma (M = 128 rows, N = Nb, K = 8) sums 8 such outer products;
// the accumulator D stays in tensor memory for the whole sweep of the tile.
//
// Shared-memory layout of the input tile ("slabs", K-major, no swizzle):
// slab s holds columns 4s..4s+3 of every tile row, one 16-byte row after the
// other.  This is the tcgen05 canonical no-swizzle layout with SBO = 128 B
// (8 rows) and LBO = slab size, so the operand for line a is the same
// descriptor moved by a*16 bytes: the row shift every coefficient line needs
// costs nothing (the paper's data-alignment conflict, Sec. 4.3, does not
// arise).  TMA brings each tile in row-major (160-byte box rows); the pass
// that splits it into TF32 parts also transposes it into slabs.
//
// Precision: TF32 (one product) or TF32x3 (a = a_hi + a_lo, h = h_hi + h_lo,
// products lo*hi + hi*lo + hi*hi accumulated in FP32), split in shared memory
// once per tile.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "mx.h"
#include "plan.h"
#include "ptx.cuh"
#include "mxutil.cuh"

namespace stx {

namespace {

using namespace mxu;

constexpr int kPad = 4;                 // input columns left/right of the output columns
constexpr int kSlabRows = 32;           // input rows per warp slab (= TMEM lanes of one warp)
constexpr int kQuarters = 4;            // TMEM lane quarters = warp slabs per tile
constexpr int kMathWarps = 16;          // 8 split warps + 8 epilogue warps
constexpr int kRoleWarps = 8;           // warps per role: two per lane quarter
constexpr int kSubs = 2;                // warps of one role per lane quarter
constexpr int kThreads = 64 + 32 * kMathWarps;  // producer warp, MMA warp, math warps
constexpr int kMathThreads = 32 * kMathWarps;
constexpr int kMaxRawStages = 6;        // TMA ring depth (fewer where shared memory runs out)
constexpr int kTmemCols = 512;
constexpr int kSmemBudget = 227 * 1024;

// Output columns per tile (the MMA block width) for a stencil with L lines:
// 32 while both accumulator sets (2 x L x 32 columns) and both A stages fit
// the 512 TMEM columns, else 16.
template <bool BF>
__host__ __device__ constexpr int a_stage_cols(int nb) {
    return OpFmt<BF>::kMaxParts * OpFmt<BF>::part_cols(OpFmt<BF>::window(nb));
}
template <bool BF>
__host__ __device__ constexpr int tile_nb(int L) { return (2 * L * 32 + 2 * a_stage_cols<BF>(32) <= kTmemCols) ? 32 : 16; }

struct MxArgs2D {
    float* out;
    const float* in;          // source grid (periodic halo fix-up reads it directly)
    const void* bops;         // banded operands [part][kchunk][line*NB + q][16 bytes]
    unsigned int* err;        // device error word (host-mapped)
    int ny, nx;
    int bc, nparts;            // operand parts of the input split (1..3)
    int tiles_x, tiles_total;
    uint32_t bop_bytes;        // every part
    uint32_t bpart_bytes;      // one part
    int nprod;                 // products per K step (1, 3 or 6)
};

// Shared-memory row pitch of the raw input tile: the K window widened to an
// odd number of 16-byte chunks, so that the 16-byte loads of eight
// consecutive rows (one shared-memory wavefront) fall in eight distinct bank
// groups.  The extra columns are loaded by TMA and never read.
__host__ __device__ constexpr int raw_pitch(int k) { return ((k / 4) & 1) ? k : k + 4; }
__host__ __device__ constexpr int raw_stage_bytes(int pitch) { return kQuarters * kSlabRows * pitch * 4; }

// Output staging: every epilogue warp owns two buffers of (32 - 2r) rows x
// NB/2 floats (its share of the tile), each padded to 1 KB, and writes them
// with its own TMA store.
__host__ __device__ constexpr int out_warp_bytes(int nb) { return ((32 * (nb / kSubs) * 4) + 1023) / 1024 * 1024; }
__host__ __device__ constexpr int out_bytes_2d(int nb) { return kRoleWarps * 2 * out_warp_bytes(nb); }

__host__ __device__ constexpr int window_2d(int nb, bool bf) {
    return bf ? OpFmt<true>::window(nb) : OpFmt<false>::window(nb);
}

// Banded operand bytes: every operand part of (window x N) elements.
__host__ __device__ constexpr int bop_bytes_2d(int nb, int lines, bool bf) {
    return (bf ? 3 * 2 : 2 * 4) * window_2d(nb, bf) * lines * nb;
}

__host__ __device__ constexpr int smem_fixed_2d(int nb, int lines, bool bf) {
    return 1024 /*align slack*/ + out_bytes_2d(nb) + bop_bytes_2d(nb, lines, bf) + 8 * (2 * kMaxRawStages + 16);
}

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }

// TMA ring depth: as many stages (up to kMaxRawStages) as shared memory holds.
__host__ __device__ constexpr int raw_stages_2d(int nb, int lines, bool bf) {
    return cmin(kMaxRawStages,
                (kSmemBudget - smem_fixed_2d(nb, lines, bf)) / raw_stage_bytes(raw_pitch(window_2d(nb, bf))));
}

__host__ __device__ constexpr int smem_bytes_2d(int nb, int lines, bool bf) {
    return smem_fixed_2d(nb, lines, bf) + raw_stages_2d(nb, lines, bf) * raw_stage_bytes(raw_pitch(window_2d(nb, bf)));
}

// Persistent, warp-specialised sweep (R = order; NB = output columns per tile).
//  * Warp 0 streams input tiles with TMA into a ring of shared-memory buffers.
//    A tile is four overlapping 32-row slabs (one per TMEM lane quarter) of
//    NB + 8 columns; slab q covers input rows Y0 + q*(32-2R) - R + [0, 32).
//  * Warps 2..9 (two per lane quarter) split their slab into TF32 hi and lo
//    parts and write them straight into tensor memory (tcgen05.st): the A
//    operand never goes back through shared memory.
//  * Warps 10..17 (two per lane quarter) drain finished accumulators and write
//    the outputs, concurrently with the split of later tiles.
//  * Warp 1 issues the outer products.  All 2R+1 coefficient lines of the
//    stencil sit side by side along N (B = [H_0 | ... | H_2R], N = NB (2R+1)),
//    so one tcgen05.mma applies every line to the same input rows; line a's
//    partial sums land in columns a*NB .. a*NB+NB-1.  The row shift a - R of
//    each line is applied in the epilogue with warp shuffles, which is why
//    each 32-row warp slab yields 32 - 2R output rows.
//  * Accuracy: TF32x3 products are accumulated corrections first (lo*hi,
//    hi*lo) and the large hi*hi products last, so each line accumulator sees
//    only (NB+8)/8 large additions (the tensor core's FP32 accumulation
//    truncates); the lines are summed in FP32 round-to-nearest in the
//    epilogue.
template <int R, int NB, bool BF>
__global__ void __launch_bounds__(kThreads, 1)
mx2d_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap_out,
            const MxArgs2D args) {
    using F = OpFmt<BF>;
    constexpr int L = 2 * R + 1;            // lines
    constexpr int N = L * NB;               // MMA N
    constexpr int K = F::window(NB);        // input columns per tile = K window
    constexpr int KS = K / F::kKStep;       // MMAs per window and product
    constexpr int ROWS_OUT = kSlabRows - 2 * R;
    constexpr int PC = F::part_cols(K);     // TMEM columns of one operand part
    constexpr int A_COLS = F::kMaxParts * PC;  // TMEM columns of one A stage
    constexpr int CW = NB / kSubs;          // epilogue columns per epilogue warp
    constexpr int GW = F::kGroup;           // input columns per split group
    constexpr int NG = K / GW;              // split groups of the input tile
    constexpr int KP = raw_pitch(K);        // shared-memory row pitch of the raw tile
    constexpr int RSB = raw_stage_bytes(KP);
    constexpr int kRawStages = raw_stages_2d(NB, L, BF);
    constexpr uint32_t SLAB_BOX = (uint32_t)(kSlabRows * KP * 4);
    static_assert(kRawStages >= 3, "TMA ring too shallow");
    static_assert(2 * A_COLS + 2 * N <= kTmemCols, "TMEM budget");

    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int OWB = out_warp_bytes(NB);
    unsigned char* outs = smem;                               // [epilogue warp][2] output buffers (1 KB aligned)
    unsigned char* raw = outs + out_bytes_2d(NB);             // kRawStages tiles
    unsigned char* bops = raw + kRawStages * RSB;
    uint64_t* bars = (uint64_t*)(bops + args.bop_bytes);
    uint64_t* full = bars;                          // [kRawStages] TMA landed
    uint64_t* rawfree = bars + kRawStages;          // [kRawStages] slab read by its math warps
    uint64_t* afull = bars + 2 * kRawStages;        // [2] A operand stage written to TMEM
    uint64_t* aempty = afull + 2;                   // [2] MMAs done reading the A stage
    uint64_t* accf = aempty + 2;                    // [2] accumulator set ready
    uint64_t* acce = accf + 2;                      // [2] accumulator set drained
    uint64_t* bop_bar = acce + 2;
    uint32_t* tmem_slot = (uint32_t*)(bop_bar + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        // split/epilogue barriers count one (elected) arrival per warp of the role
        for (int s = 0; s < kRawStages; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&rawfree[s], kRoleWarps);
        }
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(&afull[a], kRoleWarps);
            ptx::mbar_init(&aempty[a], 1);
            ptx::mbar_init(&accf[a], 1);
            ptx::mbar_init(&acce[a], kRoleWarps);
        }
        ptx::mbar_init(bop_bar, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(tmem_slot, kTmemCols);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tmem_a = tmem;                          // A stages: [2][hi | lo]
    const uint32_t tmem_d = tmem + (uint32_t)(2 * A_COLS);  // accumulator sets: [2][N]
    int issued = 0;        // producer: TMA tiles issued
    int committed = -1;    // MMA issuer: last tile whose MMAs were committed

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            ptx::mbar_arrive_expect_tx(bop_bar, args.bop_bytes);
            ptx::bulk_load(bops, args.bops, args.bop_bytes, bop_bar);
            int i = 0;
            for (int t = blockIdx.x; t < args.tiles_total; t += gridDim.x, ++i) {
                const int s = i % kRawStages;
                const uint32_t ph = (uint32_t)(i / kRawStages) & 1u;
                if (!wait_or_abort(&rawfree[s], ph ^ 1u, abort_flag)) break;
                const int X0 = (t % args.tiles_x) * NB;
                const int Y0 = (t / args.tiles_x) * (kQuarters * ROWS_OUT);
                unsigned char* dst = raw + s * RSB;
                ptx::mbar_arrive_expect_tx(&full[s], (uint32_t)kQuarters * SLAB_BOX);
#pragma unroll
                for (int q = 0; q < kQuarters; ++q)
                    ptx::tma_load_2d(dst + q * SLAB_BOX, &tmap, X0 - kPad, Y0 + q * ROWS_OUT - R, &full[s]);
                issued = i + 1;
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0 && wait_or_abort(bop_bar, 0, abort_flag)) {
            constexpr uint32_t idesc = ptx::instr_desc(F::kFmt, F::kFmt, 128, (uint32_t)N);
            const uint64_t b0 = ptx::smem_desc(ptx::smem_u32(bops), (uint32_t)(N * 16), 128);
            const int pr = args.nprod;
            int i = 0;
            for (int t = blockIdx.x; t < args.tiles_total; t += gridDim.x, ++i) {
                const int st = i & 1;
                const uint32_t ph = (uint32_t)(i >> 1) & 1u;
                if (!wait_or_abort(&afull[st], ph, abort_flag)) break;
                if (!wait_or_abort(&acce[st], ph ^ 1u, abort_flag)) break;
                ptx::tc_fence_after();
                issue_products<BF, KS>(tmem_d + (uint32_t)(st * N), tmem_a + (uint32_t)(st * A_COLS), PC, b0,
                                       args.bpart_bytes, N, idesc, pr);
                ptx::mma_commit(&aempty[st]);
                ptx::mma_commit(&accf[st]);
                committed = i;
            }
        }
    } else {
        // ------------------------------------------------ math warps
        const int q = warp & 3;                        // TMEM lane quarter (= warp slab) of this warp
        const bool split_role = (warp - 2) < kRoleWarps;
        const int sub = ((warp - 2) >> 2) & 1;         // which half of the role's work this warp takes
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        if (split_role) {
            // ---------------- split: raw tile (smem) -> TF32 hi/lo A operand (TMEM)
            int i = 0;
            for (int t = blockIdx.x; t < args.tiles_total; t += gridDim.x, ++i) {
                const int rs = i % kRawStages;
                const uint32_t rph = (uint32_t)(i / kRawStages) & 1u;
                const int st = i & 1;
                const uint32_t ph = (uint32_t)(i >> 1) & 1u;
                if (!wait_or_abort(&full[rs], rph, abort_flag) || !wait_or_abort(&aempty[st], ph ^ 1u, abort_flag))
                    break;
                ptx::tc_fence_after();
                const int X0 = (t % args.tiles_x) * NB;
                const int Y0 = (t / args.tiles_x) * (kQuarters * ROWS_OUT);
                const int gy = Y0 + q * ROWS_OUT - R + lane;   // input row of this thread
                const bool fix = (args.bc == kBcPeriodic) &&
                                 (gy < 0 || gy >= args.ny || X0 - kPad < 0 || X0 - kPad + K > args.nx);
                const float* row = reinterpret_cast<const float*>(raw + rs * RSB) + (size_t)(q * kSlabRows + lane) * KP;
                const uint32_t abase = tmem_a + lane_off + (uint32_t)(st * A_COLS);
#pragma unroll
                for (int g0 = 0; g0 < NG; g0 += kSubs) {
                    const int g = g0 + sub;
                    if (g >= NG) break;
                    const int c0 = GW * g;
                    float x[GW];
#pragma unroll
                    for (int c4 = 0; c4 < GW; c4 += 4) {
                        float4 v = *reinterpret_cast<const float4*>(row + c0 + c4);
                        if (fix) {
                            const int gx = X0 - kPad + c0 + c4;
                            if (gy < 0 || gy >= args.ny || gx < 0 || gx >= args.nx)
                                v = *reinterpret_cast<const float4*>(args.in + wrap_index(gy, args.ny) * args.nx +
                                                                     wrap_index(gx, args.nx));
                        }
                        x[c4] = v.x;
                        x[c4 + 1] = v.y;
                        x[c4 + 2] = v.z;
                        x[c4 + 3] = v.w;
                    }
                    split_store<BF>(x, abase, PC, c0, args.nparts);
                }
                ptx::tmem_wait_st();
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    ptx::mbar_arrive(&rawfree[rs]);
                    ptx::mbar_arrive(&afull[st]);
                }
            }
        } else {
            // ---------------- epilogue: accumulators (TMEM) -> row shifts -> outputs (global)
            int i = 0;
            for (int t = blockIdx.x; t < args.tiles_total; t += gridDim.x, ++i) {
                const int st = i & 1;
                const uint32_t ph = (uint32_t)(i >> 1) & 1u;
                if (!wait_or_abort(&accf[st], ph, abort_flag)) break;
                ptx::tc_fence_after();
                const int X0 = (t % args.tiles_x) * NB;
                const int Y0 = (t / args.tiles_x) * (kQuarters * ROWS_OUT);
                // this warp's CW of the tile's NB columns, for every line
                const uint32_t dbase = tmem_d + lane_off + (uint32_t)(st * N + CW * sub);
                uint32_t v[L][CW];
#pragma unroll
                for (int a = 0; a < L; ++a) {
                    if constexpr (CW == 16) {
                        ptx::tmem_ld_32x32b_x16(dbase + (uint32_t)(a * NB), v[a]);
                    } else {
                        ptx::tmem_ld_32x32b_x8(dbase + (uint32_t)(a * NB), v[a]);
                    }
                }
                ptx::tmem_wait_ld();
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&acce[st]);   // accumulators are in registers: the set is free
                float acc[CW];
#pragma unroll
                for (int c = 0; c < CW; ++c) acc[c] = __uint_as_float(v[R][c]);
#pragma unroll
                for (int a = 0; a < L; ++a) {
                    if (a == R) continue;
                    const int src = (lane + a - R) & 31;  // row this line's partial comes from
#pragma unroll
                    for (int c = 0; c < CW; ++c) acc[c] += __shfl_sync(0xffffffffu, __uint_as_float(v[a][c]), src);
                }
                // Stage this warp's outputs (its CW columns of the quarter's
                // 32 - 2R rows) row-major in its own buffer with the TMA
                // swizzle (16-byte chunk index XOR row bits; conflict-free
                // 16-byte stores), then write them with one TMA store.
                unsigned char* ost = outs + ((warp - 2 - kRoleWarps) * 2 + st) * OWB;
                if (lane == 0) ptx::bulk_wait_group_read<1>();   // this buffer's store of two tiles ago
                __syncwarp();
                if (lane >= R && lane < kSlabRows - R) {
                    const int orow = lane - R;
#pragma unroll
                    for (int c = 0; c < CW; c += 4) {
                        const int chunk = c >> 2;
                        const int sw = (CW == 16) ? (chunk ^ ((orow >> 1) & 3)) : (chunk ^ ((orow >> 2) & 1));
                        *reinterpret_cast<float4*>(ost + orow * (CW * 4) + sw * 16) =
                            make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
                    }
                }
                ptx::fence_proxy_async_smem();
                __syncwarp();
                const int ox = X0 + CW * sub, oy = Y0 + q * ROWS_OUT;
                if (lane == 0 && ox < args.nx && oy < args.ny) {
                    ptx::tma_store_2d(&tmap_out, ox, oy, ost);
                    ptx::bulk_commit_group();
                }
            }
        }
    }

    // ---- teardown (also after an abort: every role has left its loop)
    if (warp >= 2 + kRoleWarps && lane == 0) ptx::bulk_wait_group<0>();   // output stores complete
    if (*abort_flag) {
        // Let copies and MMAs still in flight land before the CTA gives up its
        // shared and tensor memory (each wait bounded again).
        if (warp == 0 && lane == 0) {
            for (int k = issued - kRawStages; k < issued; ++k)
                if (k >= 0) ptx::mbar_wait(&full[k % kRawStages], (uint32_t)(k / kRawStages) & 1u, kWaitCycles / 8);
        }
        if (warp == 1 && lane == 0 && committed >= 0)
            ptx::mbar_wait(&accf[committed & 1], (uint32_t)(committed >> 1) & 1u, kWaitCycles / 8);
    }
    __syncwarp();
    if (tid == 0 && *abort_flag) atomicOr(args.err, 1u);
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, kTmemCols);
    }
}

template <int R, bool BF>
constexpr auto kernel_for() {
    return mx2d_kernel<R, tile_nb<BF>(2 * R + 1), BF>;
}

// ------------------------------------------------------------------ host side
// Row-major 2D view of the grid; one box is a 32-row slab of an input tile
// (pitch columns: the K window, widened to an odd number of 16-byte chunks).
bool encode_tile_map_2d(CUtensorMap* map, const float* base, int ny, int nx, int pitch) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    cuuint64_t strides[1] = {(cuuint64_t)nx * 4};
    cuuint32_t box[2] = {(cuuint32_t)pitch, (cuuint32_t)kSlabRows};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Row-major 2D view of the output grid; one box is one epilogue warp's share
// of a tile (NB/2 columns x (32-2r) rows), written from shared memory with the
// TMA 64-byte (16 columns) or 32-byte (8 columns) swizzle.
bool encode_out_map_2d(CUtensorMap* map, float* base, int ny, int nx, int cols, int rows) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    cuuint64_t strides[1] = {(cuuint64_t)nx * 4};
    cuuint32_t box[2] = {(cuuint32_t)cols, (cuuint32_t)rows};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, cols == 16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

using MxKernel = void (*)(CUtensorMap, CUtensorMap, MxArgs2D);

MxKernel kernel_for_radius(int r, bool bf) {
    switch (r) {
        case 1: return bf ? kernel_for<1, true>() : kernel_for<1, false>();
        case 2: return bf ? kernel_for<2, true>() : kernel_for<2, false>();
        case 3: return bf ? kernel_for<3, true>() : kernel_for<3, false>();
        case 4: return bf ? kernel_for<4, true>() : kernel_for<4, false>();
    }
    return nullptr;
}

struct MxState {
    unsigned int* err_host = nullptr;  // host-mapped error word
    unsigned int* err_dev = nullptr;
    int num_sms = 0;
    int nb = 32;          // output columns per tile
    int in_w = 40;        // input columns per tile (the K window)
    bool bf = false;      // BF16 operands (else TF32)
    uint32_t bop_bytes = 0;
    uint32_t bpart_bytes = 0;
};

}  // namespace

bool mx_supported(const MxRequest& q, std::string* why) {
    if (q.f64) {
        if (why) *why = "FP64 storage runs on the CUDA-core kernel (no FP64 tensor-core path on this GPU)";
        return false;
    }
    if (q.ndim == 3) return mx3d_supported(q, why);
    if (q.prec < STENCIL_PREC_TF32 || q.prec > STENCIL_PREC_BF16X3) {
        if (why) *why = "the outer-product kernels run TF32, TF32X3, BF16, BF16X2 or BF16X3";
        return false;
    }
    if (q.n[1] % 4 != 0) {
        if (why) *why = "the contiguous extent must be a multiple of 4 (16-byte TMA rows)";
        return false;
    }
    if (q.tb > 1) {
        if (why) *why = "temporal blocking not built for the matrixized kernel";
        return false;
    }
    return true;
}

stencil_status mx_plan_build(const MxRequest& q, MxPlan* p, std::string* why) {
    if (!mx_supported(q, why)) return STENCIL_EUNSUPPORTED;
    p->ndim = q.ndim;
    for (int d = 0; d < 3; ++d) p->n[d] = q.n[d];
    p->r = q.r;
    p->bc = q.bc;
    p->prec = q.prec;
    p->tb = 1;
    if (q.ndim == 3) return mx3d_plan_build(q, p, why);
    const int W = 2 * q.r + 1;
    const int L = W;            // every row a of C^g is one line along the contiguous axis
    const bool bf = is_bf16(q.prec);
    const int NB = bf ? tile_nb<true>(L) : tile_nb<false>(L);
    const int KW = bf ? OpFmt<true>::window(NB) : OpFmt<false>::window(NB);
    p->nb = NB;
    std::vector<const double*> lines;
    for (int a = 0; a < L; ++a) lines.push_back(q.cg + a * W);
    uint32_t bpart = 0;
    std::vector<unsigned char> ops = pack_bands(q.r, lines, NB, KW, bf, &bpart);
    p->n_lines = L;
    p->n_scalar = 0;
    p->operand_bytes = ops.size();
    cudaError_t e = cudaMalloc(&p->d_operands, p->operand_bytes);
    if (e != cudaSuccess) {
        if (why) *why = std::string("operand upload: ") + cudaGetErrorString(e);
        return STENCIL_ENOMEM;
    }
    e = cudaMemcpy(p->d_operands, ops.data(), p->operand_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->d_operands);
        p->d_operands = nullptr;
        if (why) *why = std::string("operand upload: ") + cudaGetErrorString(e);
        return STENCIL_ECUDA;
    }
    MxState* st = new MxState();
    st->bop_bytes = (uint32_t)p->operand_bytes;
    st->bpart_bytes = bpart;
    st->nb = NB;
    st->in_w = KW;
    st->bf = bf;
    e = cudaHostAlloc((void**)&st->err_host, sizeof(unsigned int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&st->err_dev, st->err_host, 0);
    if (e != cudaSuccess) {
        cudaFree(p->d_operands);
        p->d_operands = nullptr;
        delete st;
        if (why) *why = std::string("error word: ") + cudaGetErrorString(e);
        return STENCIL_ECUDA;
    }
    *st->err_host = 0;
    p->tmap_storage = st;
    int dev = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&st->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        mx_plan_free(p);
        if (why) *why = std::string("device query: ") + cudaGetErrorString(e);
        return STENCIL_ECUDA;
    }
    if (st->bop_bytes != (uint32_t)bop_bytes_2d(NB, L, bf)) {
        mx_plan_free(p);
        if (why) *why = "internal error: banded operand size";
        return STENCIL_EUNSUPPORTED;
    }
    const size_t smem = smem_bytes_2d(NB, L, bf);
    e = cudaFuncSetAttribute(kernel_for_radius(q.r, bf), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        mx_plan_free(p);
        if (why) *why = std::string("shared memory: ") + cudaGetErrorString(e);
        return STENCIL_ECUDA;
    }
    return STENCIL_OK;
}

void mx_plan_free(MxPlan* p) {
    if (p->ndim == 3) {
        mx3d_plan_free(p);
        return;
    }
    if (p->d_operands) cudaFree(p->d_operands);
    p->d_operands = nullptr;
    MxState* st = (MxState*)p->tmap_storage;
    if (st) {
        if (st->err_host) cudaFreeHost(st->err_host);
        delete st;
    }
    p->tmap_storage = nullptr;
}

unsigned int mx_device_error(const MxPlan& p) {
    if (p.ndim == 3) return mx3d_device_error(p);
    const MxState* st = (const MxState*)p.tmap_storage;
    return st && st->err_host ? *(volatile unsigned int*)st->err_host : 0u;
}

cudaError_t mx_sweep(const MxPlan& p, const void* src, void* dst, int tb, cudaStream_t s) {
    if (p.ndim == 3) return mx3d_sweep(p, src, dst, tb, s);
    if (tb != 1) return cudaErrorInvalidValue;
    if (((uintptr_t)src & 15u) || ((uintptr_t)dst & 15u)) return cudaErrorMisalignedAddress;
    const MxState* st = (const MxState*)p.tmap_storage;
    const int ny = (int)p.n[0], nx = (int)p.n[1];
    MxArgs2D a;
    memset(&a, 0, sizeof(a));
    a.out = (float*)dst;
    a.in = (const float*)src;
    a.bops = p.d_operands;
    a.err = st->err_dev;
    a.ny = ny;
    a.nx = nx;
    a.bc = p.bc;
    a.nparts = operand_parts(p.prec);
    a.nprod = products_for(p.prec);
    a.bpart_bytes = st->bpart_bytes;
    const int in_w = st->in_w;
    a.tiles_x = (nx + st->nb - 1) / st->nb;
    const int tile_rows = kQuarters * (kSlabRows - 2 * p.r);   // output rows per tile
    a.tiles_total = a.tiles_x * ((ny + tile_rows - 1) / tile_rows);
    a.bop_bytes = st->bop_bytes;
    alignas(64) CUtensorMap map;
    alignas(64) CUtensorMap map_out;
    if (!encode_tile_map_2d(&map, (const float*)src, ny, nx, raw_pitch(in_w))) return cudaErrorInvalidValue;
    if (!encode_out_map_2d(&map_out, (float*)dst, ny, nx, st->nb / kSubs, kSlabRows - 2 * p.r))
        return cudaErrorInvalidValue;
    const int grid = a.tiles_total < st->num_sms ? a.tiles_total : st->num_sms;
    const int L = 2 * p.r + 1;
    kernel_for_radius(p.r, st->bf)<<<grid, kThreads, smem_bytes_2d(st->nb, L, st->bf), s>>>(map, map_out, a);
    return cudaGetLastError();
}

}  // namespace stx
