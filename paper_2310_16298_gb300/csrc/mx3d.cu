// Matrixized 3D stencil sweep on tcgen05 tensor cores.
//
// The grid is swept plane by plane along the slowest axis z, following the
// structure of Algorithm 1: every input plane is loaded once and scattered to
// the 2R+1 output planes it contributes to.  Within a plane the coefficient
// lines run along the contiguous axis x: line (a, b) holds the weights
// C^g[a][b][*] (a = z offset, b = y offset) as a banded operand H_ab, exactly
// as the 2D kernel uses one line per y offset.  All lines of the stencil sit
// side by side along the MMA's N dimension, so one tcgen05.mma (128 rows x
// N x 8) applies every line to one input plane; the epilogue then shifts each
// line's partial sums by b - R rows (warp shuffles) and adds them, in FP32
// round-to-nearest registers, to the running sum of output plane
// z - (a - R).  When input plane z has been scattered, output plane z - R is
// complete and is written with one TMA store.
//
// Work unit = (32-row-slab tile in y, NB columns in x, a chunk of output
// planes in z); the unit streams its chunk plus R halo planes on either side.
// Boundaries: the zero Dirichlet halo is TMA's out-of-bounds fill; with a
// periodic boundary the producer wraps the plane index (whole planes), and the
// terms that wrap in x or y are added afterwards by the edge kernel
// (edges.cu) over the boundary strips.
// Roles per CTA as in the 2D kernel: TMA producer warp, two MMA issuer warps
// (alternate input planes), 8 split warps (input plane -> TF32 hi/lo A
// operand in tensor memory), 8 epilogue warps (tensor memory -> plane
// accumulators -> TMA store).  Work units are handed out at run time from a
// per-plan atomic counter that the last CTA to finish resets.
#include <cuda.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "mx.h"
#include "mxutil.cuh"
#include "plan.h"
#include "ptx.cuh"

namespace stx {

namespace {

using namespace mxu;

constexpr int kPad = 4;
constexpr int kSlabRows = 32;
constexpr int kQuarters = 4;
constexpr int kRoleWarps = 8;
constexpr int kSubs = 2;
constexpr int kMathWarps = 2 * kRoleWarps;
constexpr int kMma2Warp = 2 + kMathWarps;   // second MMA issuer (items alternate between warps 1 and 18)
constexpr int kThreads = 32 * (kMma2Warp + 1);
constexpr int kMaxRawStages = 6;
constexpr int kUnitRing = 8;                // unit ids handed from the producer to the epilogue
constexpr int kTmemCols = 512;
constexpr int kSmemBudget = 227 * 1024;
constexpr int kChunk = 32;  // output planes per work unit (library choice; plans may set their own)

// Coefficient lines of a 3D stencil: (a = z offset, b = y offset) pairs that
// carry weights.  Box: all (2R+1)^2 pairs.  Star, parallel cover: (a, R) for
// a != R and (R, b) for every b; the centre weight sits on line (R, R).
// Star, hybrid cover (HYB): two tensor-core lines, the contiguous-axis line
// (R, R) and an identity band that hands the input rows to the epilogue, which
// applies the 4R off-axis weights to them on the CUDA cores.
template <int R, bool STAR, bool HYB = false>
struct Lines3 {
    static constexpr int W = 2 * R + 1;
    static constexpr int L = HYB ? 2 : STAR ? (4 * R + 1) : W * W;
    __host__ __device__ static constexpr int a(int l) {
        return STAR ? (l < R ? l : (l < R + W ? R : l - W + 1)) : l / W;
    }
    __host__ __device__ static constexpr int b(int l) { return STAR ? (l < R || l >= R + W ? R : l - R) : l % W; }
};

template <bool BF>
__host__ __device__ constexpr int a_stage_cols3(int nb) {
    return OpFmt<BF>::kMaxParts * OpFmt<BF>::part_cols(OpFmt<BF>::window(nb));
}
// Output columns per tile: 32 where the lines' accumulators fit twice beside
// two A stages, else 16, else 8 (the 125-point box: 25 lines).
template <bool BF>
__host__ __device__ constexpr int tile_nb3(int L) {
    return (L * 32 <= 256 && 2 * L * 32 + 2 * a_stage_cols3<BF>(32) <= kTmemCols) ? 32 : (L * 16 <= 256 ? 16 : 8);
}
// Lines as the MMA sees them: N = lines x nb must be a multiple of 16 (M =
// 128), so an odd line count at 8 columns gets one all-zero line.
__host__ __device__ constexpr int mma_lines3(int L, int nb) { return ((L * nb + 15) / 16) * 16 / nb; }
// Raw plane slabs: K window widened to an odd number of 16-byte chunks
// (conflict-free 16-byte row loads, as in the 2D kernel).
__host__ __device__ constexpr int raw_pitch3(int k) { return ((k / 4) & 1) ? k : k + 4; }
__host__ __device__ constexpr int raw_stage_bytes3(int pitch) { return kQuarters * kSlabRows * pitch * 4; }
// Output staging: two buffers of 32 rows x NB/2 floats per epilogue warp.
__host__ __device__ constexpr int out_warp_bytes3(int nb) { return ((32 * (nb / kSubs) * 4) + 1023) / 1024 * 1024; }
__host__ __device__ constexpr int out_bytes3(int nb) { return kRoleWarps * 2 * out_warp_bytes3(nb); }
__host__ __device__ constexpr int window3(int nb, bool bf) {
    return bf ? OpFmt<true>::window(nb) : OpFmt<false>::window(nb);
}
__host__ __device__ constexpr int bop_bytes3(int nb, int lines, bool bf) {
    return (bf ? 3 * 2 : 2 * 4) * window3(nb, bf) * lines * nb;
}
__host__ __device__ constexpr int smem_fixed3(int nb, int lines, bool bf) {
    return 1024 + out_bytes3(nb) + bop_bytes3(nb, lines, bf) + 8 * (2 * kMaxRawStages + 16) + 8 * 2 * kUnitRing +
           4 * (kUnitRing + kMaxRawStages + 8);
}
__host__ __device__ constexpr int raw_stages3(int nb, int lines, bool bf) {
    return (kSmemBudget - smem_fixed3(nb, lines, bf)) / raw_stage_bytes3(raw_pitch3(window3(nb, bf))) < kMaxRawStages
               ? (kSmemBudget - smem_fixed3(nb, lines, bf)) / raw_stage_bytes3(raw_pitch3(window3(nb, bf)))
               : kMaxRawStages;
}
__host__ __device__ constexpr int smem_bytes_3d(int nb, int lines, bool bf) {
    return smem_fixed3(nb, lines, bf) + raw_stages3(nb, lines, bf) * raw_stage_bytes3(raw_pitch3(window3(nb, bf)));
}

struct MxArgs3D {
    int bc;               // periodic: input planes wrap in z (x and y: edges.cu)
    const void* bops;     // banded operands [part][kchunk][line*NB + q][16 bytes]
    unsigned int* err;    // device error word (host-mapped)
    int* sched;           // [0] next unit to hand out, [1] CTAs finished (both 0 between launches)
    int nz, ny, nx;
    int64_t ldx;          // row stride of the grids (elements); planes are ny rows
    int nparts;           // operand parts of the input split (1..3)
    int tiles_x, tiles_y, chunks, units;
    int chunk;            // output planes per work unit
    uint32_t bop_bytes;
    uint32_t bpart_bytes;
    int nprod;
    float sw[12];         // hybrid cover: z weights (a != R), then y weights (b != R)
};

template <int R, bool STAR, int NB, bool BF, bool HYB>
__global__ void __launch_bounds__(kThreads, 1)
mx3d_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap_out,
            const MxArgs3D args) {
    using LN = Lines3<R, STAR, HYB>;
    static_assert(!HYB || (STAR && 4 * R <= 12), "hybrid cover: star stencils, r <= 3");
    using F = OpFmt<BF>;
    constexpr int L = LN::L;
    constexpr int LM = mma_lines3(L, NB);   // lines on the MMA (L, or L + 1 zero line)
    constexpr int N = LM * NB;
    constexpr int K = F::window(NB);
    constexpr int KS = K / F::kKStep;
    constexpr int GW = F::kGroup;
    constexpr int NG = K / GW;
    constexpr int ROWS_OUT = kSlabRows - 2 * R;
    constexpr int PC = F::part_cols(K);
    constexpr int A_COLS = F::kMaxParts * PC;
    constexpr int CW = NB / kSubs;
    constexpr int KP = raw_pitch3(K);
    constexpr int RSB = raw_stage_bytes3(KP);
    constexpr int kRawStages = raw_stages3(NB, LM, BF);
    constexpr int OWB = out_warp_bytes3(NB);
    const int PLANES = args.chunk + 2 * R;  // input planes per work unit
    constexpr uint32_t SLAB_BOX = (uint32_t)(kSlabRows * KP * 4);
    static_assert(kRawStages >= 3, "TMA ring too shallow");
    static_assert(N <= 256 && N % 16 == 0, "MMA N");
    // A stages hide the split -> MMA -> completion -> split round trip,
    // accumulator sets the MMA -> epilogue -> MMA one (as many as TMEM holds)
    constexpr int AST = (4 * A_COLS + 2 * N <= kTmemCols) ? 4 : (3 * A_COLS + 2 * N <= kTmemCols) ? 3 : 2;
    constexpr int DST = (AST * A_COLS + 3 * N <= kTmemCols) ? 3 : 2;
    static_assert(AST * A_COLS + DST * N <= kTmemCols, "TMEM budget");
    static_assert(2 * kRawStages + 2 * AST + 2 * DST + 1 <= 2 * kMaxRawStages + 15, "barrier space");

    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* outs = smem;
    unsigned char* raw = outs + out_bytes3(NB);
    unsigned char* bops = raw + kRawStages * RSB;
    uint64_t* bars = (uint64_t*)(bops + args.bop_bytes);
    uint64_t* full = bars;
    uint64_t* rawfree = bars + kRawStages;
    uint64_t* afull = bars + 2 * kRawStages;   // [AST]
    uint64_t* aempty = afull + AST;            // [AST]
    uint64_t* accf = aempty + AST;             // [DST]
    uint64_t* acce = accf + DST;               // [DST]
    uint64_t* bop_bar = acce + DST;
    uint64_t* uq_full = bop_bar + 1;           // [kUnitRing] unit id written
    uint64_t* uq_empty = uq_full + kUnitRing;  // [kUnitRing] unit id read by the epilogue warps
    uint32_t* tmem_slot = (uint32_t*)(uq_empty + kUnitRing);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    volatile int* unit_ring = abort_flag + 1;               // [kUnitRing] unit ids (-1: no more units)
    volatile int* stage_unit = unit_ring + kUnitRing;       // [kRawStages] unit of each input plane stage
    volatile int* a_unit = stage_unit + kMaxRawStages;      // [AST] -1 marks the end for the MMA issuers

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < kRawStages; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&rawfree[s], kRoleWarps);
        }
        for (int a = 0; a < AST; ++a) {
            ptx::mbar_init(&afull[a], kRoleWarps);
            ptx::mbar_init(&aempty[a], 1);
        }
        for (int a = 0; a < DST; ++a) {
            ptx::mbar_init(&accf[a], 1);
            ptx::mbar_init(&acce[a], kRoleWarps);
        }
        ptx::mbar_init(bop_bar, 1);
        for (int k = 0; k < kUnitRing; ++k) {
            ptx::mbar_init(&uq_full[k], 1);
            ptx::mbar_init(&uq_empty[k], kRoleWarps);
        }
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
    const uint32_t tmem_a = tmem;
    const uint32_t tmem_d = tmem + (uint32_t)(AST * A_COLS);
    int issued = 0, committed = -1;

    // unit u -> (x tile, y tile, z chunk), x fastest
    auto unit_origin = [&](int u, int& X0, int& Y0, int& Z0) {
        X0 = (u % args.tiles_x) * NB;
        Y0 = ((u / args.tiles_x) % args.tiles_y) * (kQuarters * ROWS_OUT);
        Z0 = (u / (args.tiles_x * args.tiles_y)) * args.chunk;
    };

    if (warp == 0) {
        if (lane == 0) {
            ptx::mbar_arrive_expect_tx(bop_bar, args.bop_bytes);
            ptx::bulk_load(bops, args.bops, args.bop_bytes, bop_bar);
            // programmatic dependent launch: grids and the unit counter only from here
            ptx::grid_dependency_wait();
            int i = 0;
            bool ok = true;
            for (int k = 0; ok; ++k) {
                const int uq = k % kUnitRing;
                if (!wait_or_abort(&uq_empty[uq], ((uint32_t)(k / kUnitRing) & 1u) ^ 1u, abort_flag)) break;
                int u = atomicAdd(&args.sched[0], 1);
                if (u >= args.units) u = -1;
                unit_ring[uq] = u;
                ptx::mbar_arrive(&uq_full[uq]);
                if (u < 0) {   // no more units: the split warps see the end through the next stage
                    const int s = i % kRawStages;
                    if (wait_or_abort(&rawfree[s], ((uint32_t)(i / kRawStages) & 1u) ^ 1u, abort_flag)) {
                        stage_unit[s] = -1;
                        ptx::mbar_arrive(&full[s]);
                    }
                    break;
                }
                int X0, Y0, Z0;
                unit_origin(u, X0, Y0, Z0);
                for (int iz = 0; iz < PLANES; ++iz, ++i) {
                    const int s = i % kRawStages;
                    const uint32_t ph = (uint32_t)(i / kRawStages) & 1u;
                    if (!wait_or_abort(&rawfree[s], ph ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    int gz = Z0 - R + iz;
                    if (args.bc == kBcPeriodic) gz = (int)wrap_index(gz, args.nz);
                    stage_unit[s] = u;
                    unsigned char* dst = raw + s * RSB;
                    ptx::mbar_arrive_expect_tx(&full[s], (uint32_t)kQuarters * SLAB_BOX);
#pragma unroll
                    for (int q = 0; q < kQuarters; ++q)
                        ptx::tma_load_3d(dst + q * SLAB_BOX, &tmap, X0 - kPad, Y0 + q * ROWS_OUT - R, gz,
                                         &full[s]);
                    issued = i + 1;
                }
            }
        }
    } else if (warp == 1 || warp == kMma2Warp) {
        // two issuers, alternating items: one issuer's barrier waits overlap the
        // other's MMAs (a thread issuing tcgen05.mma is held at the pipe's rate)
        if (lane == 0 && wait_or_abort(bop_bar, 0, abort_flag)) {
            constexpr uint32_t idesc = ptx::instr_desc(F::kFmt, F::kFmt, 128, (uint32_t)N);
            const uint64_t b0 = ptx::smem_desc(ptx::smem_u32(bops), (uint32_t)(N * 16), 128);
            const int pr = args.nprod;
            for (int i = (warp == 1 ? 0 : 1);; i += 2) {
                const int sa = i % AST;
                const uint32_t pa = (uint32_t)(i / AST) & 1u;
                const int st = i % DST;
                const uint32_t ph = (uint32_t)(i / DST) & 1u;
                if (!wait_or_abort(&afull[sa], pa, abort_flag)) break;
                if (a_unit[sa] < 0) break;   // the split warps passed the last unit
                if (!wait_or_abort(&acce[st], ph ^ 1u, abort_flag)) break;
                ptx::tc_fence_after();
                issue_products<BF, KS>(tmem_d + (uint32_t)(st * N), tmem_a + (uint32_t)(sa * A_COLS), PC, b0,
                                       args.bpart_bytes, N, idesc, pr);
                ptx::mma_commit(&aempty[sa]);
                ptx::mma_commit(&accf[st]);
                committed = i;
            }
        }
    } else {
        const int q = warp & 3;
        const bool split_role = (warp - 2) < kRoleWarps;
        const int sub = ((warp - 2) >> 2) & 1;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        int i = 0;
        bool ok = true;
        if (split_role) {
            for (;; ++i) {
                {
                    const int rs = i % kRawStages;
                    const uint32_t rph = (uint32_t)(i / kRawStages) & 1u;
                    const int sa = i % AST;
                    const uint32_t pa = (uint32_t)(i / AST) & 1u;
                    if (!wait_or_abort(&full[rs], rph, abort_flag) || !wait_or_abort(&aempty[sa], pa ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    if (stage_unit[rs] < 0) {
                        // end of the units: one end marker per MMA issuer (items i, i + 1)
                        for (int e2 = 0; e2 < 2; ++e2) {
                            const int sb = (i + e2) % AST;
                            if (e2 == 1 &&
                                !wait_or_abort(&aempty[sb], ((uint32_t)((i + 1) / AST) & 1u) ^ 1u, abort_flag))
                                break;
                            if (warp == 2 && lane == 0) a_unit[sb] = -1;
                            __syncwarp();
                            if (lane == 0) ptx::mbar_arrive(&afull[sb]);
                        }
                        break;
                    }
                    ptx::tc_fence_after();
                    const float* row = reinterpret_cast<const float*>(raw + rs * RSB) + (size_t)(q * kSlabRows + lane) * KP;
                    const uint32_t abase = tmem_a + lane_off + (uint32_t)(sa * A_COLS);
#pragma unroll
                    for (int g0 = 0; g0 < NG; g0 += kSubs) {
                        const int g = g0 + sub;
                        if (g >= NG) break;
                        const int c0 = GW * g;
                        float x[GW];
#pragma unroll
                        for (int c4 = 0; c4 < GW; c4 += 4) {
                            const float4 v = *reinterpret_cast<const float4*>(row + c0 + c4);
                            x[c4] = v.x;
                            x[c4 + 1] = v.y;
                            x[c4 + 2] = v.z;
                            x[c4 + 3] = v.w;
                        }
                        split_store<BF>(x, abase, PC, c0, args.nparts);
                    }
                    ptx::tc_fence_before();
                    if (warp == 2 && lane == 0) a_unit[sa] = 0;
                    __syncwarp();
                    if (lane == 0) {
                        ptx::mbar_arrive(&rawfree[rs]);
                        ptx::mbar_arrive(&afull[sa]);
                    }
                }
            }
        } else {
            int nstore = 0;
            for (int k = 0; ok; ++k) {
                const int uq = k % kUnitRing;
                if (!wait_or_abort(&uq_full[uq], (uint32_t)(k / kUnitRing) & 1u, abort_flag)) break;
                const int u = unit_ring[uq];
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&uq_empty[uq]);
                if (u < 0) break;
                int X0, Y0, Z0;
                unit_origin(u, X0, Y0, Z0);
                float acc[2 * R + 1][CW];  // running sums of output planes z-R .. z+R
#pragma unroll
                for (int j = 0; j < 2 * R + 1; ++j)
#pragma unroll
                    for (int c = 0; c < CW; ++c) acc[j][c] = 0.0f;
                for (int iz = 0; iz < PLANES; ++iz, ++i) {
                    const int st = i % DST;
                    const uint32_t ph = (uint32_t)(i / DST) & 1u;
                    if (!wait_or_abort(&accf[st], ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t dbase = tmem_d + lane_off + (uint32_t)(st * N + CW * sub);
                    if constexpr (HYB) {
                        // contiguous-axis line -> centre plane; identity band (the
                        // input rows) x off-axis weights: z offsets without a row
                        // shift, y offsets shifted by b - R rows
                        uint32_t vx[CW], vi[CW];
                        if constexpr (CW == 16)
                            ptx::tmem_ld_x16_sync(dbase, vx, dbase + (uint32_t)NB, vi);
                        else
                            ptx::tmem_ld_x8_sync(dbase, vx, dbase + (uint32_t)NB, vi);
#pragma unroll
                        for (int c = 0; c < CW; ++c) acc[R][c] += __uint_as_float(vx[c]);
#pragma unroll
                        for (int k = 0; k < 2 * R; ++k) {
                            const int a = k < R ? k : k + 1;
                            const float w = args.sw[k];
#pragma unroll
                            for (int c = 0; c < CW; ++c) acc[2 * R - a][c] += w * __uint_as_float(vi[c]);
                        }
#pragma unroll
                        for (int k = 0; k < 2 * R; ++k) {
                            const int b = k < R ? k : k + 1;
                            const float w = args.sw[2 * R + k];
                            const int src = (lane + b - R) & 31;
                            float tv[CW];
#pragma unroll
                            for (int c = 0; c < CW; ++c) tv[c] = __shfl_sync(0xffffffffu, __uint_as_float(vi[c]), src);
#pragma unroll
                            for (int c = 0; c < CW; ++c) acc[R][c] += w * tv[c];
                        }
                    } else {
                        // line (a, b): rows shift by b - R, target output plane slot 2R - a.
                        // Lines are drained in batches of LB to bound live registers.
                        constexpr int LB = (CW == 16) ? 2 : 4;
                        static_assert(CW == 16 || CW == 8 || CW == 4, "epilogue column share");
    #pragma unroll
                        for (int l0 = 0; l0 < L; l0 += LB) {
                            uint32_t v[LB][CW];
                            const int nv = L - l0 < LB ? L - l0 : LB;   // lines in this batch
                            const uint32_t ba = dbase + (uint32_t)(l0 * NB);
                            if constexpr (CW == 16) {
                                if (nv == 2) ptx::tmem_ld_x16_sync(ba, v[0], ba + NB, v[1]);
                                if (nv == 1) ptx::tmem_ld_x16_sync(ba, v[0]);
                            } else if constexpr (CW == 4) {
                                if (nv == 4)
                                    ptx::tmem_ld_x4_sync(ba, v[0], ba + NB, v[1], ba + 2 * NB, v[2], ba + 3 * NB, v[3]);
                                if (nv == 3) ptx::tmem_ld_x4_sync(ba, v[0], ba + NB, v[1], ba + 2 * NB, v[2]);
                                if (nv == 2) ptx::tmem_ld_x4_sync(ba, v[0], ba + NB, v[1]);
                                if (nv == 1) ptx::tmem_ld_x4_sync(ba, v[0]);
                            } else {
                                if constexpr (LB >= 4) {
                                    if (nv == 4)
                                        ptx::tmem_ld_x8_sync(ba, v[0], ba + NB, v[1], ba + 2 * NB, v[2], ba + 3 * NB, v[3]);
                                    if (nv == 3) ptx::tmem_ld_x8_sync(ba, v[0], ba + NB, v[1], ba + 2 * NB, v[2]);
                                }
                                if (nv == 2) ptx::tmem_ld_x8_sync(ba, v[0], ba + NB, v[1]);
                                if (nv == 1) ptx::tmem_ld_x8_sync(ba, v[0]);
                            }
    #pragma unroll
                            for (int j = 0; j < LB; ++j) {
                                const int l = l0 + j;
                                if (l < L) {
                                    const int la = LN::a(l), lb = LN::b(l);
                                    const int src = (lane + lb - R) & 31;
    #pragma unroll
                                    for (int c = 0; c < CW; ++c) {
                                        const float val = (lb == R) ? __uint_as_float(v[j][c])
                                                                    : __shfl_sync(0xffffffffu, __uint_as_float(v[j][c]), src);
                                        acc[2 * R - la][c] += val;
                                    }
                                }
                            }
                        }
                    }
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&acce[st]);
                    if (iz >= 2 * R) {
                        // output plane Z0 + iz - 2R is complete: this warp stages its
                        // share (swizzled, conflict-free) and stores it with one TMA store
                        unsigned char* ost = outs + ((warp - 2 - kRoleWarps) * 2 + (nstore & 1)) * OWB;
                        if (lane == 0) ptx::bulk_wait_group_read<1>();
                        __syncwarp();
                        if (lane >= R && lane < kSlabRows - R) {
                            const int orow = lane - R;
#pragma unroll
                            for (int c = 0; c < CW; c += 4) {
                                const int chunk = c >> 2;
                                // the output map's swizzle: 64B for 64-byte rows, 32B for
                                // 32-byte rows, none for 16-byte rows
                                const int sw = (CW == 16)  ? (chunk ^ ((orow >> 1) & 3))
                                               : (CW == 8) ? (chunk ^ ((orow >> 2) & 1))
                                                           : chunk;
                                *reinterpret_cast<float4*>(ost + orow * (CW * 4) + sw * 16) =
                                    make_float4(acc[0][c], acc[0][c + 1], acc[0][c + 2], acc[0][c + 3]);
                            }
                        }
                        ptx::fence_proxy_async_smem();
                        __syncwarp();
                        const int ox = X0 + CW * sub, oy = Y0 + q * ROWS_OUT;
                        if (lane == 0 && ox < args.nx && oy < args.ny && Z0 + iz - 2 * R < args.nz) {
                            ptx::tma_store_3d(&tmap_out, ox, oy, Z0 + iz - 2 * R, ost);
                            ptx::bulk_commit_group();
                        }
                        ++nstore;
                    }
                    // slide the window of output planes by one
#pragma unroll
                    for (int j = 0; j < 2 * R; ++j)
#pragma unroll
                        for (int c = 0; c < CW; ++c) acc[j][c] = acc[j + 1][c];
#pragma unroll
                    for (int c = 0; c < CW; ++c) acc[2 * R][c] = 0.0f;
                }
            }
        }
    }

    // output stores have read their staging buffers (the writes are visible to
    // later work in the stream once the grid completes)
    if (warp >= 2 + kRoleWarps && warp < kMma2Warp && lane == 0) ptx::bulk_wait_group_read<0>();
    if (*abort_flag) {
        if (warp == 0 && lane == 0) {
            for (int k = issued - kRawStages; k < issued; ++k)
                if (k >= 0) ptx::mbar_wait(&full[k % kRawStages], (uint32_t)(k / kRawStages) & 1u, kWaitCycles / 8);
        }
        if ((warp == 1 || warp == kMma2Warp) && lane == 0 && committed >= 0)
            ptx::mbar_wait(&accf[committed % DST], (uint32_t)(committed / DST) & 1u, kWaitCycles / 8);
    }
    __syncwarp();
    if (tid == 0 && *abort_flag) atomicOr(args.err, 1u);
    ptx::tc_fence_before();
    __syncthreads();
    if (tid == 0) {   // this CTA's producer is done: the last CTA resets the unit counter
        __threadfence();
        if (atomicAdd(&args.sched[1], 1) == (int)gridDim.x - 1) {
            atomicExch(&args.sched[0], 0);
            atomicExch(&args.sched[1], 0);
        }
    }
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, kTmemCols);
    }
}

using Mx3Kernel = void (*)(CUtensorMap, CUtensorMap, MxArgs3D);

// Output columns per tile: tile_nb3 of the line count, except that the hybrid
// cover's 2r+1 register plane sums stay within the register budget only at
// 16 columns for r >= 2.
template <bool BF>
__host__ __device__ constexpr int nb3(int r, int lines, bool hyb) {
    return (hyb && r >= 2) ? 16 : tile_nb3<BF>(lines);
}

template <int R, bool STAR, bool BF, bool HYB>
Mx3Kernel kernel3() {
    return mx3d_kernel<R, STAR, nb3<BF>(R, Lines3<R, STAR, HYB>::L, HYB), BF, HYB>;
}

template <int R>
Mx3Kernel kernel3_star(bool bf, bool hyb) {
    if (hyb) return bf ? kernel3<R, true, true, true>() : kernel3<R, true, false, true>();
    return bf ? kernel3<R, true, true, false>() : kernel3<R, true, false, false>();
}

// Kernel for order r, star/box, BF16 (else TF32) operands, hybrid star cover.
Mx3Kernel kernel3_for(int r, bool star, bool bf, bool hyb) {
    if (star) {
        switch (r) {
            case 1: return kernel3_star<1>(bf, hyb);
            case 2: return kernel3_star<2>(bf, hyb);
            case 3: return kernel3_star<3>(bf, hyb);
        }
    } else if (!hyb) {
        if (r == 1) return bf ? kernel3<1, false, true, false>() : kernel3<1, false, false, false>();
        if (r == 2) return bf ? kernel3<2, false, true, false>() : kernel3<2, false, false, false>();
    }
    return nullptr;
}

// Tensor-core lines of a plan (hybrid star cover: the contiguous-axis line
// and the identity band).
int lines3(int r, bool star, bool hyb = false) {
    return hyb ? 2 : star ? 4 * r + 1 : (2 * r + 1) * (2 * r + 1);
}
int line3_a(int r, bool star, int l) {
    const int W = 2 * r + 1;
    return star ? (l < r ? l : (l < r + W ? r : l - W + 1)) : l / W;
}
int line3_b(int r, bool star, int l) {
    const int W = 2 * r + 1;
    return star ? (l < r || l >= r + W ? r : l - r) : l % W;
}

bool encode_in_map_3d(CUtensorMap* map, const float* base, int nz, int ny, int nx, int64_t ldx, int pitch) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[2] = {(cuuint64_t)ldx * 4, (cuuint64_t)ldx * ny * 4};
    cuuint32_t box[3] = {(cuuint32_t)pitch, (cuuint32_t)kSlabRows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One box = one epilogue warp's share of an output plane tile (cols = NB/2).
bool encode_out_map_3d(CUtensorMap* map, float* base, int nz, int ny, int nx, int64_t ldx, int cols, int rows) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[2] = {(cuuint64_t)ldx * 4, (cuuint64_t)ldx * ny * 4};
    cuuint32_t box[3] = {(cuuint32_t)cols, (cuuint32_t)rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE,
               cols == 16 ? CU_TENSOR_MAP_SWIZZLE_64B : cols == 8 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct Mx3State {
    unsigned int* err_host = nullptr;
    unsigned int* err_dev = nullptr;
    int* sched = nullptr;  // device unit counter pair (zero between launches)
    int num_sms = 0;
    int nb = 16;
    int in_w = 24;
    bool star = false;
    bool bf = false;
    bool hyb = false;     // hybrid star cover
    float sw[12] = {};    // its off-axis weights (z, then y)
    uint32_t bop_bytes = 0;
    uint32_t bpart_bytes = 0;
};

// The hybrid cover is the library's choice for 3D stars.
bool use_hybrid(const MxRequest& q) { return q.star && q.cover != STENCIL_COVER_PARALLEL; }

}  // namespace

bool mx3d_supported(const MxRequest& q, std::string* why) {
    if (!mx_precision(q.prec)) {
        if (why) *why = "the outer-product kernels run TF32, TF32X3, BF16, BF16X2, BF16X3 or BF16_W2";
        return false;
    }
    if (q.cover == STENCIL_COVER_HYBRID && !q.star) {
        if (why) *why = "the hybrid line cover applies to star stencils";
        return false;
    }
    if (!kernel3_for(q.r, q.star, false, use_hybrid(q))) {
        if (why) *why = "3D matrixized kernel built for 7/13/19-point stars (r <= 3) and the 27- and 125-point boxes";
        return false;
    }
    if (q.ldx % 4 != 0) {
        if (why) *why = "the row stride must be a multiple of 4 (16-byte TMA rows)";
        return false;
    }
    if (q.tb > 1) {
        if (why) *why = "temporal blocking not built for the matrixized kernel";
        return false;
    }
    return true;
}

stencil_status mx3d_plan_build(const MxRequest& q, MxPlan* p, std::string* why) {
    if (!mx3d_supported(q, why)) return STENCIL_EUNSUPPORTED;
    const int r = q.r, W = 2 * r + 1;
    const bool hyb = use_hybrid(q);
    const int L = lines3(r, q.star, hyb);
    const bool bf = is_bf16(q.prec);
    const int NB = bf ? nb3<true>(r, L, hyb) : nb3<false>(r, L, hyb);
    const int KW = bf ? OpFmt<true>::window(NB) : OpFmt<false>::window(NB);
    p->nb = NB;
    std::vector<const double*> lines;
    std::vector<double> ident(W, 0.0);   // the identity band's weights: the row itself
    ident[r] = 1.0;
    if (hyb) {
        lines.push_back(q.cg + ((size_t)r * W + r) * W);   // contiguous-axis line (r, r)
        lines.push_back(ident.data());
    } else {
        for (int l = 0; l < L; ++l)
            lines.push_back(q.cg + ((size_t)line3_a(r, q.star, l) * W + line3_b(r, q.star, l)) * W);
    }
    const int LM = mma_lines3(L, NB);
    std::vector<double> zero_line(W, 0.0);   // pads N to a multiple of 16
    while ((int)lines.size() < LM) lines.push_back(zero_line.data());
    uint32_t bpart = 0;
    std::vector<unsigned char> ops = pack_bands(r, lines, NB, KW, bf, &bpart);
    p->n_lines = L;
    p->n_scalar = hyb ? 4 * r : 0;
    p->cover = hyb ? STENCIL_COVER_HYBRID : STENCIL_COVER_PARALLEL;
    p->operand_bytes = ops.size();
    cudaError_t e = cudaMalloc(&p->d_operands, p->operand_bytes);
    if (e != cudaSuccess) {
        if (why) *why = std::string("operand upload: ") + cudaGetErrorString(e);
        return STENCIL_ENOMEM;
    }
    e = cudaMemcpy(p->d_operands, ops.data(), p->operand_bytes, cudaMemcpyHostToDevice);
    Mx3State* st = new Mx3State();
    st->nb = NB;
    st->in_w = KW;
    st->star = q.star;
    st->bf = bf;
    st->hyb = hyb;
    if (hyb)
        for (int k = 0; k < 2 * r; ++k) {
            const int o = k < r ? k : k + 1;   // offsets 0..2r except r
            st->sw[k] = (float)q.cg[((size_t)o * W + r) * W + r];            // z offset o
            st->sw[2 * r + k] = (float)q.cg[((size_t)r * W + o) * W + r];    // y offset o
        }
    st->bop_bytes = (uint32_t)p->operand_bytes;
    st->bpart_bytes = bpart;
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&st->err_host, sizeof(unsigned int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&st->err_dev, st->err_host, 0);
    if (e == cudaSuccess) e = cudaMalloc(&st->sched, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(st->sched, 0, 2 * sizeof(int));
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&st->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && st->bop_bytes != (uint32_t)bop_bytes3(NB, LM, bf)) e = cudaErrorInvalidValue;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel3_for(r, q.star, bf, hyb), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_bytes_3d(NB, LM, bf));
    p->tmap_storage = st;
    if (e != cudaSuccess) {
        if (why) *why = std::string("3D plan set-up: ") + cudaGetErrorString(e);
        mx3d_plan_free(p);
        return STENCIL_ECUDA;
    }
    *st->err_host = 0;
    return STENCIL_OK;
}

void mx3d_plan_free(MxPlan* p) {
    if (p->d_operands) cudaFree(p->d_operands);
    p->d_operands = nullptr;
    Mx3State* st = (Mx3State*)p->tmap_storage;
    if (st) {
        if (st->err_host) cudaFreeHost(st->err_host);
        if (st->sched) cudaFree(st->sched);
        delete st;
    }
    p->tmap_storage = nullptr;
}

unsigned int mx3d_device_error(const MxPlan& p) {
    const Mx3State* st = (const Mx3State*)p.tmap_storage;
    return st && st->err_host ? *(volatile unsigned int*)st->err_host : 0u;
}

cudaError_t mx3d_sweep(const MxPlan& p, const void* src, void* dst, int tb, cudaStream_t s) {
    if (tb != 1) return cudaErrorInvalidValue;
    if (((uintptr_t)src & 15u) || ((uintptr_t)dst & 15u)) return cudaErrorMisalignedAddress;
    const Mx3State* st = (const Mx3State*)p.tmap_storage;
    const int nz = (int)p.n[0], ny = (int)p.n[1], nx = (int)p.n[2];
    const int in_w = st->in_w;
    const int rows_tile = kQuarters * (kSlabRows - 2 * p.r);
    MxArgs3D a;
    memset(&a, 0, sizeof(a));
    a.bc = p.bc;
    a.bops = p.d_operands;
    a.err = st->err_dev;
    a.sched = st->sched;
    a.nz = nz;
    a.ny = ny;
    a.nx = nx;
    a.ldx = p.ldx;
    a.nparts = operand_parts(p.prec);
    a.nprod = products_for(p.prec);
    a.bpart_bytes = st->bpart_bytes;
    a.tiles_x = (nx + st->nb - 1) / st->nb;
    a.tiles_y = (ny + rows_tile - 1) / rows_tile;
    a.chunk = p.unit_planes > 0 ? p.unit_planes : kChunk;
    a.chunks = (nz + a.chunk - 1) / a.chunk;
    a.units = a.tiles_x * a.tiles_y * a.chunks;
    a.bop_bytes = st->bop_bytes;
    alignas(64) CUtensorMap map, map_out;
    if (!encode_in_map_3d(&map, (const float*)src, nz, ny, nx, p.ldx, raw_pitch3(in_w))) return cudaErrorInvalidValue;
    if (!encode_out_map_3d(&map_out, (float*)dst, nz, ny, nx, p.ldx, st->nb / kSubs, kSlabRows - 2 * p.r))
        return cudaErrorInvalidValue;
    const int grid = a.units < st->num_sms ? a.units : st->num_sms;
    for (int k = 0; k < 12; ++k) a.sw[k] = st->sw[k];
    const int smem = smem_bytes_3d(st->nb, mma_lines3(lines3(p.r, st->star, st->hyb), st->nb), st->bf);
    return launch_dependent(kernel3_for(p.r, st->star, st->bf, st->hyb), grid, kThreads, smem, s, map, map_out, a);
}

}  // namespace stx
