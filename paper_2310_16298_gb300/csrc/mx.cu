// Matrixized 2D stencil sweep on the 5th-generation tensor cores (tcgen05).
//
// Scatter-mode formulation (Sec. 3): every coefficient line contributes, to
// an output block, the sum over its input vectors of (input vector) x
// (coefficient vector) outer products -- Eq. (final).  The lines run along
// the contiguous axis x (the orientation of Eq. (to-outer-product-2-star)):
// line a holds row a of C^g, i.e. the weights of input row offset a - r.  For
// an output block of NB = 16 columns starting at X0, line a applied to input
// row y is the product of the row's K window (columns X0-4 .. X0-4+W-1) with
// the line's banded Toeplitz operand
//
//     H_a[k, q] = C^g[a, k - q - 4 + r],
//
// whose columns are the coefficient vectors (windows of a column of C^o,
// Eq. (co)).  One tcgen05.mma (M = 128, N, K = 8 or 16) sums K such outer
// products for 128 rows at once; the accumulators stay in tensor memory.
//
// Row pairs.  The line sum needs, for output row Y, the partials of line a
// at input row Y + a - r: a shift across the accumulator rows (TMEM lanes),
// which only warp shuffles can apply.  To halve those shuffles every TMEM
// lane m holds two input rows, 2m (even) and 2m+1 (odd), side by side along
// K (K = 2W), and the B operand is made of 2r+2 column blocks, block (p, d)
// stacking H_{a0} over H_{a0+1} with a0 = 2d - p + r (lines outside 0..2r
// are zero).  Lane m+d of block (p, d) then holds exactly the contribution
// of its two rows to output row 2m+p, so
//
//     B[2m + p, :] = sum_d D[m + d, block (p, d)],     |d| <= ceil(r/2),
//
// r shuffles per output instead of 2r, and fewer MACs per output than one
// lane per row.
//
// Tiles are handed out at run time (an atomic counter per plan, reset by the
// last CTA to finish), so SMs that run faster take more tiles.
//
// Boundaries: rows and columns outside the grid are TMA's out-of-bounds zero
// fill (the zero Dirichlet halo); with a periodic boundary the terms that
// wrap are added afterwards by the edge kernel (edges.cu).
//
// Roles (one persistent CTA per SM, warp specialised):
//  * warp 0: TMA producer.  A tile is 4 lane quarters x 64 input rows; each
//    quarter is loaded as two 32-row boxes through row-parity tensor maps
//    (even rows, odd rows), so a warp reads consecutive rows (no bank
//    conflicts) and every lane's two rows sit in the same smem slot.
//  * warps 1 and 18: MMA issuers (one thread each), alternating items.  A
//    thread issuing tcgen05.mma is held at the tensor pipe's rate, so with
//    one issuer the pipe drains while that thread waits on the next item's
//    barriers; with two, one issuer's waits overlap the other's MMAs.
//  * warps 2..9: split warps, one per (quarter, row parity): input rows ->
//    TF32 hi/lo (or BF16 parts) -> tensor memory (tcgen05.st).
//  * warps 10..17: epilogue warps, one per (quarter, output parity): tensor
//    memory -> shuffles -> swizzled smem -> TMA store through the output
//    row-parity tensor map.
// Two or three accumulator sets and A stages (as many as tensor memory
// holds) overlap split, MMA and epilogue; every wait is bounded
// (a timeout sets a host-visible error word, drains copies in flight and
// frees tensor memory).  Every CTA loads the banded operands from one of
// several identical copies, so the CTAs starting together do not all read
// the same L2 lines.
//
// Precision: TF32, TF32x3, BF16, BF16x2, BF16x3 (operand parts products
// accumulated smallest first in FP32; the epilogue sums the blocks in FP32
// round-to-nearest).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <array>
#include <cmath>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "mx.h"
#include "mxutil.cuh"
#include "plan.h"
#include "ptx.cuh"

namespace stx {

namespace {

using namespace mxu;

constexpr int kPad = 4;                 // input columns left of the output block
constexpr int kLanes = 32;              // TMEM lanes per warp (lane quarter)
constexpr int kQuarters = 4;
constexpr int kNb = 16;                 // output columns per MMA item
constexpr int kItems = 2;               // items (16-column blocks) per tile
constexpr int kTw = kItems * kNb;       // output columns per tile
constexpr int kSplitWarps = 2 * kQuarters;   // (quarter, input row parity)
constexpr int kEpiWarps = 2 * kQuarters;     // (quarter, output row parity)
constexpr int kMma2Warp = 2 + kSplitWarps + kEpiWarps;   // second MMA issuer
constexpr int kThreads = 32 * (kMma2Warp + 1);
constexpr int kBopCopies = 16;          // copies of the banded operands in global memory
constexpr int kMaxRawStages = 6;
constexpr int kTileRing = 8;            // tile ids handed from the producer to the epilogue
constexpr int kTmemCols = 512;
constexpr int kSmemBudget = 227 * 1024;

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }

// Row-pair geometry of order R.
template <int R>
struct Pair {
    static constexpr int DM = (R + 1) / 2;              // lanes an output row reaches on either side
    static constexpr int LANES_OUT = kLanes - 2 * DM;   // lanes of a quarter that produce outputs
    static constexpr int ROWS_OUT = 2 * LANES_OUT;      // output rows per quarter
    static constexpr int NBP = R + 1;                   // blocks per output parity
    static constexpr int NBLK = 2 * NBP;
    // lane offset d of block (p, i) is dlo(p) + i
    __host__ __device__ static constexpr int dlo(int p) { return -((R + 1 - p) / 2); }
};

template <bool BF>
__host__ __device__ constexpr int window(int nb) { return BF ? OpFmt<true>::window(nb) : OpFmt<false>::window(nb); }

// Shared-memory row pitch of the raw tile: the window widened to an odd
// number of 16-byte chunks (eight consecutive rows = eight bank groups).
__host__ __device__ constexpr int raw_pitch(int w) { return ((w / 4) & 1) ? w : w + 4; }
// Raw tile row: the windows of all items of a tile (item j starts 16 j columns in).
template <bool BF>
__host__ __device__ constexpr int raw_row(int nb) { return nb * (kItems - 1) + window<BF>(nb); }
template <bool BF>
__host__ __device__ constexpr int raw_stage_bytes() { return 2 * kQuarters * kLanes * raw_pitch(raw_row<BF>(kNb)) * 4; }

// Output staging: one buffer per epilogue warp of (32 - 2 DM) rows x kTw floats
// (both items of a tile, written with one TMA store).
__host__ __device__ constexpr int out_warp_bytes() { return 32 * kTw * 4; }
__host__ __device__ constexpr int out_bytes() { return kEpiWarps * out_warp_bytes(); }

template <int R, bool BF>
__host__ __device__ constexpr int bop_bytes() {
    return (BF ? 3 * 2 : 2 * 4) * 2 * window<BF>(kNb) * Pair<R>::NBLK * kNb;
}
template <int R, bool BF>
__host__ __device__ constexpr int smem_fixed() {
    return 1024 /*align slack*/ + out_bytes() + bop_bytes<R, BF>() + 8 * (2 * kMaxRawStages + 16) +
           8 * 2 * kTileRing + 4 * (kTileRing + kMaxRawStages + 8);
}
template <int R, bool BF>
__host__ __device__ constexpr int raw_stages() {
    return cmin(kMaxRawStages, (kSmemBudget - smem_fixed<R, BF>()) / raw_stage_bytes<BF>());
}
template <int R, bool BF>
__host__ __device__ constexpr int smem_bytes() {
    return smem_fixed<R, BF>() + raw_stages<R, BF>() * raw_stage_bytes<BF>();
}

struct MxArgs2D {
    const void* bops;          // block operands [part][kchunk][block*16 + q][16 bytes]
    unsigned int* err;         // device error word (host-mapped)
    int* sched;                // [0] next tile to hand out, [1] CTAs finished (both 0 between launches)
    int ny, nx;
    int64_t ldx;               // row stride of the grids (elements)
    int nparts;                // operand parts of the input split (1..3)
    int tiles_x, tiles_total;
    int rows_even, rows_odd;   // rows of the even / odd row-parity views
    uint32_t bop_bytes;        // every part
    uint32_t bpart_bytes;      // one part
    int nprod;                 // products per K step (1, 3 or 6)
};

// Tensor-memory stage counts for A operands of a_cols columns and
// accumulator sets of n columns: as many A stages as fit (up to 4) beside two
// accumulator sets, then as many accumulator sets as fit beside those.
__host__ __device__ constexpr int a_stages(int a_cols, int n) {
    return (4 * a_cols + 2 * n <= kTmemCols) ? 4 : (3 * a_cols + 2 * n <= kTmemCols) ? 3 : 2;
}
__host__ __device__ constexpr int d_sets(int a_cols, int n) {
    return (a_stages(a_cols, n) * a_cols + 4 * n <= kTmemCols)   ? 4
           : (a_stages(a_cols, n) * a_cols + 3 * n <= kTmemCols) ? 3
                                                                 : 2;
}

template <int R, bool BF, int NP>
__global__ void __launch_bounds__(kThreads, 1)
mx2d_kernel(const __grid_constant__ CUtensorMap tmap_e, const __grid_constant__ CUtensorMap tmap_o,
            const __grid_constant__ CUtensorMap omap_e, const __grid_constant__ CUtensorMap omap_o,
            const MxArgs2D args) {
    using F = OpFmt<BF>;
    using G = Pair<R>;
    constexpr int N = G::NBLK * kNb;        // MMA N
    constexpr int W = window<BF>(kNb);      // K window of one input row
    constexpr int KW = 2 * W;               // K: even-row window | odd-row window
    constexpr int KS = KW / F::kKStep;      // MMAs per product
    constexpr int PC = F::part_cols(KW);    // TMEM columns of one operand part
    constexpr int A_COLS = NP * PC;         // NP operand parts (1..3) per A stage
    constexpr int GW = F::kGroup;           // input columns per split group
    constexpr int NG = W / GW;              // split groups per row
    constexpr int KP = raw_pitch(raw_row<BF>(kNb));
    constexpr int SLAB = kLanes * KP * 4;   // one (parity, quarter) box
    constexpr int RSB = raw_stage_bytes<BF>();
    constexpr int kRawStages = raw_stages<R, BF>();
    constexpr int OWB = out_warp_bytes();
    // A stages hide the split -> MMA -> completion -> split round trip,
    // accumulator sets the MMA -> epilogue -> MMA one
    constexpr int AST = a_stages(A_COLS, N);
    constexpr int DST = d_sets(A_COLS, N);
    static_assert(kRawStages * kItems >= 4, "TMA ring too shallow");
    static_assert(N % 16 == 0 && N <= 256, "MMA N");
    static_assert(2 * A_COLS + 2 * N <= kTmemCols, "TMEM budget");
    static_assert(AST * A_COLS + DST * N <= kTmemCols, "TMEM budget");
    static_assert(2 * kRawStages + 2 * AST + 2 * DST + 1 <= 2 * kMaxRawStages + 15, "barrier space");
    static_assert(G::LANES_OUT * kTw * 4 <= OWB && kTw * 4 == 128, "output staging (128-byte swizzle rows)");

    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* outs = smem;                     // [epilogue warp] output buffers (1 KB aligned)
    unsigned char* raw = outs + out_bytes();        // [stage][parity][quarter] 32-row boxes
    unsigned char* bops = raw + kRawStages * RSB;
    uint64_t* bars = (uint64_t*)(bops + args.bop_bytes);
    uint64_t* full = bars;                          // [kRawStages] TMA landed
    uint64_t* rawfree = bars + kRawStages;          // [kRawStages] rows read by the split warps
    uint64_t* afull = bars + 2 * kRawStages;        // [AST] A operand stage written to TMEM
    uint64_t* aempty = afull + AST;                 // [AST] MMAs done reading the A stage
    uint64_t* accf = aempty + AST;                  // [DST] accumulator set ready
    uint64_t* acce = accf + DST;                    // [DST] accumulator set drained
    uint64_t* bop_bar = acce + DST;
    uint64_t* tq_full = bop_bar + 1;                // [kTileRing] tile id written
    uint64_t* tq_empty = tq_full + kTileRing;       // [kTileRing] tile id read by the epilogue warps
    uint32_t* tmem_slot = (uint32_t*)(tq_empty + kTileRing);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    volatile int* tile_ring = abort_flag + 1;       // [kTileRing] tile ids (-1: no more tiles)
    volatile int* stage_tile = tile_ring + kTileRing;   // [kRawStages] tile of each input stage
    volatile int* a_tile = stage_tile + kMaxRawStages;  // [AST] tile of each A stage (-1: end)

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < kRawStages; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&rawfree[s], kSplitWarps);
        }
        for (int a = 0; a < AST; ++a) {
            ptx::mbar_init(&afull[a], kSplitWarps);
            ptx::mbar_init(&aempty[a], 1);
        }
        for (int a = 0; a < DST; ++a) {
            ptx::mbar_init(&accf[a], 1);
            ptx::mbar_init(&acce[a], kEpiWarps);
        }
        ptx::mbar_init(bop_bar, 1);
        for (int k = 0; k < kTileRing; ++k) {
            ptx::mbar_init(&tq_full[k], 1);
            ptx::mbar_init(&tq_empty[k], kEpiWarps);
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
    const uint32_t tmem_a = tmem;                             // A stages: [AST][parts]
    const uint32_t tmem_d = tmem + (uint32_t)(AST * A_COLS);  // accumulator sets: [DST][N]
    int issued = 0;        // producer: TMA tiles issued
    int committed = -1;    // MMA issuer: last tile whose MMAs were committed

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            ptx::mbar_arrive_expect_tx(bop_bar, args.bop_bytes);
            ptx::bulk_load(bops, (const unsigned char*)args.bops + (size_t)(blockIdx.x % kBopCopies) * args.bop_bytes,
                           args.bop_bytes, bop_bar);
            // Launched as a programmatic dependent of the stream's previous
            // kernel (the previous sweep, or its boundary-strip kernel): the
            // set-up above (barriers, tensor memory, banded operands) overlapped
            // its tail; the grids and the tile counter are touched only from here.
            ptx::grid_dependency_wait();
            for (int i = 0;; ++i) {
                const int s = i % kRawStages;
                const uint32_t ph = (uint32_t)(i / kRawStages) & 1u;
                const int tq = i % kTileRing;
                if (!wait_or_abort(&rawfree[s], ph ^ 1u, abort_flag) ||
                    !wait_or_abort(&tq_empty[tq], ((uint32_t)(i / kTileRing) & 1u) ^ 1u, abort_flag))
                    break;
                int t = atomicAdd(&args.sched[0], 1);
                if (t >= args.tiles_total) t = -1;
                stage_tile[s] = t;
                tile_ring[tq] = t;
                ptx::mbar_arrive(&tq_full[tq]);
                if (t < 0) {   // no more tiles: the split warps see the end through the stage
                    ptx::mbar_arrive(&full[s]);
                    break;
                }
                const int X0 = (t % args.tiles_x) * kTw;
                const int Y0 = (t / args.tiles_x) * (kQuarters * G::ROWS_OUT);
                unsigned char* dst = raw + s * RSB;
                ptx::mbar_arrive_expect_tx(&full[s], (uint32_t)RSB);
#pragma unroll
                for (int q = 0; q < kQuarters; ++q) {
                    // quarter q covers input rows Y0 + q*ROWS_OUT - 2*DM + [0, 64): an even start
                    const int yp = (Y0 + q * G::ROWS_OUT - 2 * G::DM) / 2;   // row in the parity views
                    ptx::tma_load_2d(dst + q * SLAB, &tmap_e, X0 - kPad, yp, &full[s]);
                    ptx::tma_load_2d(dst + (kQuarters + q) * SLAB, &tmap_o, X0 - kPad, yp, &full[s]);
                }
                issued = i + 1;
            }
        }
    } else if (warp == 1 || warp == kMma2Warp) {
        // ------------------------------------------------ MMA issuers (items i with i % 2 == u)
        const int u = warp == 1 ? 0 : 1;
        if (lane == 0 && wait_or_abort(bop_bar, 0, abort_flag)) {
            constexpr uint32_t idesc = ptx::instr_desc(F::kFmt, F::kFmt, 128, (uint32_t)N);
            const uint64_t b0 = ptx::smem_desc(ptx::smem_u32(bops), (uint32_t)(N * 16), 128);
            const int pr = args.nprod;
            for (int i = u;; i += 2) {
                const int sa = i % AST;
                const uint32_t pa = (uint32_t)(i / AST) & 1u;
                const int st = i % DST;
                const uint32_t ph = (uint32_t)(i / DST) & 1u;
                if (!wait_or_abort(&afull[sa], pa, abort_flag)) break;
                if (a_tile[sa] < 0) break;   // the split warps passed the end of the tiles
                if (!wait_or_abort(&acce[st], ph ^ 1u, abort_flag)) break;
                ptx::tc_fence_after();
                issue_products<BF, KS>(tmem_d + (uint32_t)(st * N), tmem_a + (uint32_t)(sa * A_COLS), PC, b0,
                                       args.bpart_bytes, N, idesc, pr);
                ptx::mma_commit(&aempty[sa]);
                ptx::mma_commit(&accf[st]);
                committed = i;
            }
        }
    } else if (warp < 2 + kSplitWarps) {
        // ------------------------------------------------ split: rows (smem) -> operand parts (TMEM)
        const int q = warp & 3;                        // TMEM lane quarter of this warp
        const int e = (warp - 2) >> 2;                 // input row parity this warp converts
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        int i = 0;   // items
        bool ok = true;
        for (int k = 0; ok; ++k) {
            const int rs = k % kRawStages;
            const uint32_t rph = (uint32_t)(k / kRawStages) & 1u;
            if (!wait_or_abort(&full[rs], rph, abort_flag)) break;
            const int t = stage_tile[rs];
            if (t < 0) {
                // End of the tiles: one end marker per MMA issuer through the
                // next two A stages (the issuers take alternate items).
                for (int e2 = 0; e2 < 2; ++e2, ++i) {
                    const int sa = i % AST;
                    if (!wait_or_abort(&aempty[sa], ((uint32_t)(i / AST) & 1u) ^ 1u, abort_flag)) break;
                    if (warp == 2 && lane == 0) a_tile[sa] = -1;
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&afull[sa]);
                }
                break;
            }
            const float* row =
                reinterpret_cast<const float*>(raw + rs * RSB + (e * kQuarters + q) * SLAB) + (size_t)lane * KP;
            for (int j = 0; j < kItems; ++j, ++i) {
                const int sa = i % AST;
                const uint32_t pa = (uint32_t)(i / AST) & 1u;
                float x[NG][GW];
#pragma unroll
                for (int g = 0; g < NG; ++g) {
#pragma unroll
                    for (int c4 = 0; c4 < GW; c4 += 4) {
                        const float4 v = *reinterpret_cast<const float4*>(row + kNb * j + GW * g + c4);
                        x[g][c4] = v.x;
                        x[g][c4 + 1] = v.y;
                        x[g][c4 + 2] = v.z;
                        x[g][c4 + 3] = v.w;
                    }
                }
                if (j == kItems - 1) {   // every item's rows are in registers: the stage goes back
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&rawfree[rs]);
                }
                if (!wait_or_abort(&aempty[sa], pa ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t abase = tmem_a + lane_off + (uint32_t)(sa * A_COLS);
                split_store_groups<BF, NP, NG>(x, abase, PC, e * W, GW);
                ptx::tc_fence_before();
                if (warp == 2 && lane == 0) a_tile[sa] = t;
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&afull[sa]);
            }
        }
    } else {
        // ------------------------------------------------ epilogue: accumulators -> outputs (warps 10..17)
        const int q = warp & 3;
        const int p = (warp - 2 - kSplitWarps) >> 2;   // output row parity of this warp
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        unsigned char* ost = outs + (warp - 2 - kSplitWarps) * OWB;
        auto drain = [&](auto pc) {
            constexpr int P = decltype(pc)::value;
            constexpr int DLO = G::dlo(P);
            constexpr int I0 = -DLO;                          // the block with lane offset 0
            constexpr int LB = G::NBP <= 3 ? G::NBP : 2;      // blocks per TMEM load batch
            const CUtensorMap* omap = P ? &omap_o : &omap_e;
            const int prows = P ? args.rows_odd : args.rows_even;
            int i = 0;
            bool ok = true;
            for (int k = 0; ok; ++k) {
            const int tq = k % kTileRing;
            if (!wait_or_abort(&tq_full[tq], (uint32_t)(k / kTileRing) & 1u, abort_flag)) break;
            const int t = tile_ring[tq];
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&tq_empty[tq]);
            if (t < 0) break;
            for (int j = 0; j < kItems; ++j, ++i) {
                const int st = i % DST;
                const uint32_t ph = (uint32_t)(i / DST) & 1u;
                if (!wait_or_abort(&accf[st], ph, abort_flag)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const int X0 = (t % args.tiles_x) * kTw;
                const int Y0 = (t / args.tiles_x) * (kQuarters * G::ROWS_OUT);
                const uint32_t dbase = tmem_d + lane_off + (uint32_t)(st * N + P * G::NBP * kNb);
                float acc[kNb];
#pragma unroll
                for (int b0 = 0; b0 < G::NBP; b0 += LB) {
                    // Blocks b0 .. b0 + nv - 1 into v (and, with the first batch,
                    // block I0 into v0 when it lies in a later batch), loaded and
                    // waited for in one step.
                    uint32_t v[LB][kNb];
                    uint32_t v0[kNb];
                    const int nv = G::NBP - b0 < LB ? G::NBP - b0 : LB;
                    const uint32_t ba = dbase + (uint32_t)(b0 * kNb);
                    const uint32_t bi = dbase + (uint32_t)(I0 * kNb);
                    if (b0 == 0 && I0 >= LB) {
                        if (nv == 2) ptx::tmem_ld_x16_sync(ba, v[0], ba + kNb, v[1], bi, v0);
                        if (nv == 1) ptx::tmem_ld_x16_sync(ba, v[0], bi, v0);
                    } else {
                        if constexpr (LB >= 3) {
                            if (nv == 3) ptx::tmem_ld_x16_sync(ba, v[0], ba + kNb, v[1], ba + 2 * kNb, v[2]);
                        }
                        if (nv == 2) ptx::tmem_ld_x16_sync(ba, v[0], ba + kNb, v[1]);
                        if (nv == 1) ptx::tmem_ld_x16_sync(ba, v[0]);
                    }
                    if (b0 + LB >= G::NBP) {   // last batch: the accumulator set is free
                        ptx::tc_fence_before();
                        __syncwarp();
                        if (lane == 0) ptx::mbar_arrive(&acce[st]);
                    }
                    if (b0 == 0) {
                        if constexpr (I0 < LB) {
#pragma unroll
                            for (int c = 0; c < kNb; ++c) acc[c] = __uint_as_float(v[I0][c]);
                        } else {
#pragma unroll
                            for (int c = 0; c < kNb; ++c) acc[c] = __uint_as_float(v0[c]);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < LB; ++j) {
                        if (b0 + j < G::NBP && b0 + j != I0) {
                            const int src = (lane + DLO + b0 + j) & 31;   // lane m + d of this block
                            float tv[kNb];   // a block's shuffles in flight before the adds
#pragma unroll
                            for (int c = 0; c < kNb; ++c)
                                tv[c] = __shfl_sync(0xffffffffu, __uint_as_float(v[j][c]), src);
#pragma unroll
                            for (int c = 0; c < kNb; ++c) acc[c] += tv[c];
                        }
                    }
                }
                // Stage this warp's output rows (one parity of the quarter,
                // item j's 16 columns of the tile's 32) with the TMA 128-byte
                // swizzle (16-byte chunk XOR row bits), then one TMA store per
                // tile through the parity view.
                if (j == 0) {
                    if (lane == 0) ptx::bulk_wait_group_read<0>();   // the previous tile's store has read the buffer
                    __syncwarp();
                }
                if (lane >= G::DM && lane < kLanes - G::DM) {
                    const int o = lane - G::DM;
#pragma unroll
                    for (int c = 0; c < kNb; c += 4) {
                        const int sw = ((kNb * j + c) >> 2) ^ (o & 7);
                        *reinterpret_cast<float4*>(ost + o * (kTw * 4) + sw * 16) =
                            make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
                    }
                }
                if (j == kItems - 1) {
                    ptx::fence_proxy_async_smem();
                    __syncwarp();
                    const int oy = (Y0 + q * G::ROWS_OUT) / 2;   // first output row of the quarter, parity view
                    if (lane == 0 && X0 < args.nx && oy < prows) {
                        ptx::tma_store_2d(omap, X0, oy, ost);
                        ptx::bulk_commit_group();
                    }
                }
            }
            }
        };
        if (p == 0)
            drain(std::integral_constant<int, 0>{});
        else
            drain(std::integral_constant<int, 1>{});
    }

    // ---- teardown (also after an abort: every role has left its loop)
    // output stores have read their staging buffers (the writes themselves
    // are visible to later work in the stream once the grid completes)
    if (warp >= 2 + kSplitWarps && warp < kMma2Warp && lane == 0) ptx::bulk_wait_group_read<0>();
    if (*abort_flag) {
        // Let copies and MMAs still in flight land before the CTA gives up its
        // shared and tensor memory (each wait bounded again).
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
    if (tid == 0) {   // every producer of this CTA is done: the last CTA resets the tile counter
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

// ------------------------------------------------------------------ host side
using MxKernel = void (*)(CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, MxArgs2D);

struct KernelInfo {
    MxKernel fn = nullptr;
    int smem = 0;
};

template <int R, bool BF, int NP>
KernelInfo kernel_info() {
    return {mx2d_kernel<R, BF, NP>, smem_bytes<R, BF>()};
}

template <int R>
KernelInfo kernel_for_parts(bool bf, int np) {
    if (bf) return np == 1 ? kernel_info<R, true, 1>() : np == 2 ? kernel_info<R, true, 2>() : kernel_info<R, true, 3>();
    return np == 1 ? kernel_info<R, false, 1>() : kernel_info<R, false, 2>();
}

// Kernel of order r for BF16 (else TF32) operands split into np parts.
KernelInfo kernel_for(int r, bool bf, int np) {
    switch (r) {
        case 1: return kernel_for_parts<1>(bf, np);
        case 2: return kernel_for_parts<2>(bf, np);
        case 3: return kernel_for_parts<3>(bf, np);
        case 4: return kernel_for_parts<4>(bf, np);
    }
    return {};
}

// Block list of order r: block (p, i) (lane offset d = dlo(p) + i) stacks
// line 2d - p + r over line 2d - p + r + 1 (null outside 0..2r).
std::vector<std::array<const double*, 2>> pair_blocks(int r, const double* cg) {
    const int W = 2 * r + 1;
    std::vector<std::array<const double*, 2>> out;
    for (int p = 0; p < 2; ++p) {
        const int dlo = -((r + 1 - p) / 2);
        for (int i = 0; i <= r; ++i) {
            std::array<const double*, 2> b{nullptr, nullptr};
            for (int e = 0; e < 2; ++e) {
                const int a = 2 * (dlo + i) - p + r + e;
                if (a >= 0 && a <= 2 * r) b[e] = cg + a * W;
            }
            out.push_back(b);
        }
    }
    return out;
}

// Row-parity view of a row-major grid with rows of ldx elements: rows parity,
// parity + 2, ... (a 2D tensor of rows_p rows of nx elements, row stride two
// grid rows).
bool encode_parity_map(CUtensorMap* map, const float* base, int rows_p, int nx, int64_t ldx, int box_x, int box_y,
                       CUtensorMapSwizzle swz, CUtensorMapL2promotion l2) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)rows_p};
    cuuint64_t strides[1] = {(cuuint64_t)ldx * 8};
    cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, swz, l2, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct MxState {
    unsigned int* err_host = nullptr;  // host-mapped error word
    unsigned int* err_dev = nullptr;
    int* sched = nullptr;              // device tile counter pair (zero between launches)
    int num_sms = 0;
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
    if (q.cover == STENCIL_COVER_HYBRID) {
        if (why) *why = "the hybrid line cover is built for 3D stars";
        return false;
    }
    if (!mx_precision(q.prec)) {
        if (why) *why = "the outer-product kernels run TF32, TF32X3, BF16, BF16X2, BF16X3 or BF16_W2";
        return false;
    }
    if (q.ldx % 4 != 0) {
        if (why) *why = "the row stride must be a multiple of 4 (16-byte TMA rows)";
        return false;
    }
    if (q.n[0] < 2) {
        if (why) *why = "the matrixized 2D kernel needs at least two rows";
        return false;
    }
    if (q.tb > 1) {
        if (why) *why = "temporal blocking not built for the matrixized kernel";
        return false;
    }
    return true;
}

// Periodic plans also get the boundary-term table of the edge kernel; a plan
// that cannot get it is freed.
static stencil_status with_edges(const MxRequest& q, MxPlan* p, std::string* why) {
    const stencil_status s = mx_edges_build(q, p);
    if (s != STENCIL_OK) {
        mx_plan_free(p);
        if (why) *why = "the periodic boundary-term table holds r <= 4 and at most 120 terms";
    }
    return s;
}

stencil_status mx_plan_build(const MxRequest& q, MxPlan* p, std::string* why) {
    if (!mx_supported(q, why)) return STENCIL_EUNSUPPORTED;
    p->ndim = q.ndim;
    for (int d = 0; d < 3; ++d) p->n[d] = q.n[d];
    p->ldx = q.ldx;
    p->unit_planes = q.unit_planes;
    p->r = q.r;
    p->bc = q.bc;
    p->prec = q.prec;
    p->tb = 1;
    p->n_edge_terms = 0;
    if (q.ndim == 3) {
        const stencil_status s3 = mx3d_plan_build(q, p, why);
        return s3 == STENCIL_OK ? with_edges(q, p, why) : s3;
    }
    const bool bf = is_bf16(q.prec);
    const int W = bf ? window<true>(kNb) : window<false>(kNb);
    p->nb = kNb;
    const auto blocks = pair_blocks(q.r, q.cg);
    uint32_t bpart = 0;
    std::vector<unsigned char> ops = pack_blocks(q.r, blocks, kNb, W, bf, &bpart);
    p->n_lines = 2 * q.r + 1;
    p->cover = STENCIL_COVER_PARALLEL;
    p->n_scalar = 0;
    const size_t one = ops.size();   // one copy; CTA b reads copy b % kBopCopies
    p->operand_bytes = one * kBopCopies;
    const KernelInfo ki = kernel_for(q.r, bf, operand_parts(q.prec));
    if (!ki.fn || one != (size_t)(bf ? 3 : 2) * bpart || one % 16 != 0) {
        if (why) *why = "internal error: block operand size";
        return STENCIL_EUNSUPPORTED;
    }
    std::vector<unsigned char> copies(p->operand_bytes);
    for (int c = 0; c < kBopCopies; ++c) memcpy(copies.data() + c * one, ops.data(), one);
    cudaError_t e = cudaMalloc(&p->d_operands, p->operand_bytes);
    if (e != cudaSuccess) {
        if (why) *why = std::string("operand upload: ") + cudaGetErrorString(e);
        return STENCIL_ENOMEM;
    }
    e = cudaMemcpy(p->d_operands, copies.data(), p->operand_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->d_operands);
        p->d_operands = nullptr;
        if (why) *why = std::string("operand upload: ") + cudaGetErrorString(e);
        return STENCIL_ECUDA;
    }
    MxState* st = new MxState();
    st->bop_bytes = (uint32_t)one;
    st->bpart_bytes = bpart;
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
    e = cudaMalloc(&st->sched, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(st->sched, 0, 2 * sizeof(int));
    if (e != cudaSuccess) {
        mx_plan_free(p);
        if (why) *why = std::string("tile counter: ") + cudaGetErrorString(e);
        return STENCIL_ENOMEM;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&st->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(ki.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ki.smem);
    if (e != cudaSuccess) {
        mx_plan_free(p);
        if (why) *why = std::string("kernel set-up: ") + cudaGetErrorString(e);
        return STENCIL_ECUDA;
    }
    return with_edges(q, p, why);
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
        if (st->sched) cudaFree(st->sched);
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
    const cudaError_t e = p.ndim == 3 ? mx3d_sweep(p, src, dst, tb, s) : mx2d_sweep(p, src, dst, tb, s);
    // periodic boundary: the kernels ran with a zero halo in x and y
    return e == cudaSuccess ? mx_periodic_edges(p, src, dst, s) : e;
}

cudaError_t mx2d_sweep(const MxPlan& p, const void* src, void* dst, int tb, cudaStream_t s) {
    if (tb != 1) return cudaErrorInvalidValue;
    if (((uintptr_t)src & 15u) || ((uintptr_t)dst & 15u)) return cudaErrorMisalignedAddress;
    const MxState* st = (const MxState*)p.tmap_storage;
    const int ny = (int)p.n[0], nx = (int)p.n[1];
    const int dm = (p.r + 1) / 2;
    const int rows_out = 2 * (kLanes - 2 * dm);          // output rows per quarter
    const int RWD = st->bf ? raw_row<true>(kNb) : raw_row<false>(kNb);
    MxArgs2D a;
    memset(&a, 0, sizeof(a));
    a.bops = p.d_operands;
    a.err = st->err_dev;
    a.sched = st->sched;
    a.ny = ny;
    a.nx = nx;
    a.ldx = p.ldx;
    a.nparts = operand_parts(p.prec);
    a.nprod = products_for(p.prec);
    a.bpart_bytes = st->bpart_bytes;
    a.tiles_x = (nx + kTw - 1) / kTw;
    a.tiles_total = a.tiles_x * ((ny + kQuarters * rows_out - 1) / (kQuarters * rows_out));
    a.rows_even = (ny + 1) / 2;
    a.rows_odd = ny / 2;
    a.bop_bytes = st->bop_bytes;
    const float* in = (const float*)src;
    float* out = (float*)dst;
    alignas(64) CUtensorMap te, to, oe, oo;
    const int kp = raw_pitch(RWD);
    const int64_t ld = p.ldx;
    if (!encode_parity_map(&te, in, a.rows_even, nx, ld, kp, kLanes, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B) ||
        !encode_parity_map(&to, in + ld, a.rows_odd, nx, ld, kp, kLanes, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B) ||
        !encode_parity_map(&oe, out, a.rows_even, nx, ld, kTw, kLanes - 2 * dm, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_NONE) ||
        !encode_parity_map(&oo, out + ld, a.rows_odd, nx, ld, kTw, kLanes - 2 * dm, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_NONE))
        return cudaErrorInvalidValue;
    const KernelInfo ki = kernel_for(p.r, st->bf, operand_parts(p.prec));
    const int grid = a.tiles_total < st->num_sms ? a.tiles_total : st->num_sms;
    return launch_dependent(ki.fn, grid, kThreads, ki.smem, s, te, to, oe, oo, a);
}

}  // namespace stx
