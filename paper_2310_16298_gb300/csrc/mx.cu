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

namespace stx {

namespace {

constexpr int kNb = 16;                 // output columns per line per MMA block
constexpr int kPad = 4;                 // input columns left/right of the output columns
constexpr int kK = kNb + 2 * kPad;      // K window per block (24)
constexpr int kKSteps = kK / 8;         // tf32 MMAs (K = 8) per window (3)
constexpr int kKChunks = kK / 4;        // 16-byte K chunks per window (6)
constexpr int kSlabRows = 32;           // input rows per warp slab (= TMEM lanes of one warp)
constexpr int kMathWarps = 4;           // one per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kMathWarps;  // producer warp, MMA warp, math warps
constexpr int kMathThreads = 32 * kMathWarps;
constexpr int kMaxLines = 2 * kMaxRadius + 1;
constexpr int kMaxBlocks = 2;
constexpr int kMaxInW = kMaxBlocks * kNb + 2 * kPad;  // 40
constexpr int kRawStages = 6;           // TMA ring depth
constexpr int kTmemCols = 512;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

struct MxArgs2D {
    float* out;
    const float* in;          // source grid (periodic halo fix-up reads it directly)
    const float* bops;        // banded operands [part][kchunk][line*16 + q][4]
    unsigned int* err;        // device error word (host-mapped)
    int ny, nx;
    int r, bc, nlines, nprod;  // nprod: 1 (TF32) or 3 (TF32x3)
    int nblk;                  // MMA blocks (of kNb output columns) per tile
    int in_w;                  // input columns per tile: nblk*16 + 8
    int rows_out;              // output rows per warp slab: 32 - 2r
    int tiles_x, tiles_total;
    uint32_t bop_bytes;        // both parts
};

__host__ __device__ inline int raw_stage_bytes(int in_w) { return kMathWarps * kSlabRows * in_w * 4; }

size_t smem_bytes_2d(int in_w, uint32_t bop_bytes) {
    return 1024 /*align slack*/ + (size_t)kRawStages * raw_stage_bytes(in_w) + bop_bytes +
           8 * (2 * kRawStages + 16);
}

// Bounded mbarrier wait that also gives up once another role has failed.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    const long long t0 = clock64();
    while (!ptx::mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// Persistent, warp-specialised sweep.
//  * Warp 0 streams input tiles with TMA into a ring of shared-memory buffers.
//    A tile is four overlapping 32-row slabs (one per TMEM lane quarter) of
//    nblk*16 + 8 columns; slab q covers input rows Y0 + q*(32-2r) - r + [0, 32).
//  * Warps 2..5 (one per lane quarter) split their slab into TF32 hi and lo
//    parts and write them straight into tensor memory (tcgen05.st): the
//    A operand never goes back through shared memory.  One tile behind, the
//    same warps drain the accumulators and write the outputs.
//  * Warp 1 issues the outer products.  All coefficient lines of the stencil
//    sit side by side along N (B = [H_0 | H_1 | ... ], N = 16 * lines), so one
//    tcgen05.mma applies every line to the same input rows; line a's partial
//    sums land in columns a*16 .. a*16+15.  The row shift a - r of each line
//    is applied in the epilogue with warp shuffles, which is why each warp
//    slab yields 32 - 2r output rows.
//  * Accuracy: TF32x3 products are accumulated corrections first (lo*hi,
//    hi*lo) and the large hi*hi products last, so each line accumulator sees
//    only kKSteps large additions (the tensor core's FP32 accumulation
//    truncates); lines are summed in FP32 round-to-nearest in the epilogue.
__global__ void __launch_bounds__(kThreads, 1)
mx2d_kernel(const __grid_constant__ CUtensorMap tmap, const MxArgs2D args) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int in_w = args.in_w;
    const int RSB = raw_stage_bytes(in_w);
    unsigned char* raw = smem;                                // kRawStages tiles
    unsigned char* bops = raw + kRawStages * RSB;
    uint64_t* bars = (uint64_t*)(bops + args.bop_bytes);
    uint64_t* full = bars;                          // [kRawStages] TMA landed
    uint64_t* rawfree = bars + kRawStages;          // [kRawStages] slab read by its math warp
    uint64_t* afull = bars + 2 * kRawStages;        // [2] A operand stage written to TMEM
    uint64_t* aempty = afull + 2;                   // [2] MMAs done reading the A stage
    uint64_t* accf = aempty + 2;                    // [2] accumulator set ready
    uint64_t* acce = accf + 2;                      // [2] accumulator set drained
    uint64_t* bop_bar = acce + 2;
    uint32_t* tmem_slot = (uint32_t*)(bop_bar + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int r = args.r;
    const int L = args.nlines;
    const int N = L * kNb;                 // MMA N: all lines side by side
    const int a_cols = 2 * in_w;           // TMEM columns of one A stage (hi | lo)
    const int set_cols = args.nblk * N;    // TMEM columns of one accumulator set
    const uint32_t slab_box_bytes = (uint32_t)(kSlabRows * in_w * 4);

    if (tid == 0) {
        for (int s = 0; s < kRawStages; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&rawfree[s], kMathThreads);
        }
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(&afull[a], kMathThreads);
            ptx::mbar_init(&aempty[a], 1);
            ptx::mbar_init(&accf[a], 1);
            ptx::mbar_init(&acce[a], kMathThreads);
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
    const uint32_t tmem_d = tmem + (uint32_t)(2 * a_cols);  // accumulator sets: [2][nblk][N]
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
                const int X0 = (t % args.tiles_x) * (args.nblk * kNb);
                const int Y0 = (t / args.tiles_x) * (kMathWarps * args.rows_out);
                unsigned char* dst = raw + s * RSB;
                ptx::mbar_arrive_expect_tx(&full[s], (uint32_t)kMathWarps * slab_box_bytes);
                for (int q = 0; q < kMathWarps; ++q)
                    ptx::tma_load_2d(dst + q * slab_box_bytes, &tmap, X0 - kPad, Y0 + q * args.rows_out - r, &full[s]);
                issued = i + 1;
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0 && wait_or_abort(bop_bar, 0, abort_flag)) {
            const uint32_t idesc = ptx::instr_desc(2, 2, 128, (uint32_t)N);
            const uint32_t part_bytes = args.bop_bytes / 2;
            const uint64_t bhi0 = ptx::smem_desc(ptx::smem_u32(bops), (uint32_t)(N * 16), 128);
            const uint64_t blo0 = bhi0 + (uint64_t)(part_bytes >> 4);
            int i = 0;
            for (int t = blockIdx.x; t < args.tiles_total; t += gridDim.x, ++i) {
                const int st = i & 1;
                const uint32_t ph = (uint32_t)(i >> 1) & 1u;
                if (!wait_or_abort(&afull[st], ph, abort_flag)) break;
                if (!wait_or_abort(&acce[st], ph ^ 1u, abort_flag)) break;
                ptx::tc_fence_after();
                const uint32_t ahi = tmem_a + (uint32_t)(st * a_cols);
                const uint32_t alo = ahi + (uint32_t)in_w;
                for (int j = 0; j < args.nblk; ++j) {
                    const uint32_t d = tmem_d + (uint32_t)(st * set_cols + j * N);
                    const uint32_t k0 = (uint32_t)(j * kNb);
                    if (args.nprod > 1) {
#pragma unroll
                        for (int ks = 0; ks < kKSteps; ++ks) {
                            const uint64_t boff = (uint64_t)((2 * ks * N * 16) >> 4);
                            ptx::mma_tf32_ts(d, alo + k0 + 8 * ks, bhi0 + boff, idesc, ks > 0);
                        }
#pragma unroll
                        for (int ks = 0; ks < kKSteps; ++ks) {
                            const uint64_t boff = (uint64_t)((2 * ks * N * 16) >> 4);
                            ptx::mma_tf32_ts(d, ahi + k0 + 8 * ks, blo0 + boff, idesc, 1u);
                        }
                    }
#pragma unroll
                    for (int ks = 0; ks < kKSteps; ++ks) {
                        const uint64_t boff = (uint64_t)((2 * ks * N * 16) >> 4);
                        ptx::mma_tf32_ts(d, ahi + k0 + 8 * ks, bhi0 + boff, idesc, (args.nprod > 1 || ks > 0) ? 1u : 0u);
                    }
                }
                ptx::mma_commit(&aempty[st]);
                ptx::mma_commit(&accf[st]);
                committed = i;
            }
        }
    } else {
        // ------------------------------------------------ math warps: split + epilogue
        const int q = warp & 3;                  // TMEM lane quarter (= warp slab) of this warp
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        int i = 0, prev_t = -1;
        bool ok = true;
        auto epilogue = [&](int ii, int tt) -> bool {
            const int st = ii & 1;
            const uint32_t ph = (uint32_t)(ii >> 1) & 1u;
            if (!wait_or_abort(&accf[st], ph, abort_flag)) return false;
            ptx::tc_fence_after();
            const int X0 = (tt % args.tiles_x) * (args.nblk * kNb);
            const int Y0 = (tt / args.tiles_x) * (kMathWarps * args.rows_out);
            const bool valid_lane = (lane >= r) && (lane < kSlabRows - r);
            const int64_t gy = (int64_t)Y0 + q * args.rows_out + (lane - r);
            for (int j = 0; j < args.nblk; ++j) {
                const uint32_t dbase = tmem_d + lane_off + (uint32_t)(st * set_cols + j * N);
                float acc[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) acc[c] = 0.0f;
                for (int a = 0; a < L; ++a) {
                    uint32_t v[16];
                    ptx::tmem_ld_32x32b_x16(dbase + (uint32_t)(a * kNb), v);
                    ptx::tmem_wait_ld();
                    const int src = lane + a - r;  // row this line's partial comes from
#pragma unroll
                    for (int c = 0; c < 16; ++c) acc[c] += __shfl_sync(0xffffffffu, __uint_as_float(v[c]), src & 31);
                }
                if (valid_lane && gy < args.ny) {
                    float* dst = args.out + gy * args.nx + X0 + j * kNb;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if (X0 + j * kNb + 4 * c < args.nx)
                            *reinterpret_cast<float4*>(dst + 4 * c) =
                                make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
                    }
                }
            }
            ptx::tc_fence_before();
            ptx::mbar_arrive(&acce[st]);
            return true;
        };
        for (int t = blockIdx.x; t < args.tiles_total && ok; t += gridDim.x, ++i) {
            const int rs = i % kRawStages;
            const uint32_t rph = (uint32_t)(i / kRawStages) & 1u;
            const int st = i & 1;
            const uint32_t ph = (uint32_t)(i >> 1) & 1u;
            if (!wait_or_abort(&full[rs], rph, abort_flag) || !wait_or_abort(&aempty[st], ph ^ 1u, abort_flag)) {
                ok = false;
                break;
            }
            ptx::tc_fence_after();
            const int X0 = (t % args.tiles_x) * (args.nblk * kNb);
            const int Y0 = (t / args.tiles_x) * (kMathWarps * args.rows_out);
            const int gy = Y0 + q * args.rows_out - r + lane;   // input row of this thread
            const bool fix = (args.bc == kBcPeriodic) &&
                             (gy < 0 || gy >= args.ny || X0 - kPad < 0 || X0 - kPad + in_w > args.nx);
            const float* row = reinterpret_cast<const float*>(raw + rs * RSB) + (size_t)(q * kSlabRows + lane) * in_w;
            const uint32_t ahi = tmem_a + lane_off + (uint32_t)(st * a_cols);
            const uint32_t alo = ahi + (uint32_t)in_w;
            for (int c8 = 0; c8 < in_w; c8 += 8) {
                float4 v0 = *reinterpret_cast<const float4*>(row + c8);
                float4 v1 = *reinterpret_cast<const float4*>(row + c8 + 4);
                if (fix) {
                    const int64_t wy = wrap_index(gy, args.ny);
                    const int gx0 = X0 - kPad + c8;
                    if (gy < 0 || gy >= args.ny || gx0 < 0 || gx0 >= args.nx)
                        v0 = *reinterpret_cast<const float4*>(args.in + wy * args.nx + wrap_index(gx0, args.nx));
                    if (gy < 0 || gy >= args.ny || gx0 + 4 < 0 || gx0 + 4 >= args.nx)
                        v1 = *reinterpret_cast<const float4*>(args.in + wy * args.nx + wrap_index(gx0 + 4, args.nx));
                }
                const float x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                uint32_t h[8], l[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float hv = ptx::to_tf32(x[e]);
                    h[e] = __float_as_uint(hv);
                    l[e] = __float_as_uint(ptx::to_tf32(x[e] - hv));
                }
                ptx::tmem_st_32x32b_x8(ahi + (uint32_t)c8, h);
                if (args.nprod > 1) ptx::tmem_st_32x32b_x8(alo + (uint32_t)c8, l);
            }
            ptx::tmem_wait_st();
            ptx::mbar_arrive(&rawfree[rs]);
            ptx::tc_fence_before();
            ptx::mbar_arrive(&afull[st]);
            if (prev_t >= 0 && !epilogue(i - 1, prev_t)) {
                ok = false;
                break;
            }
            prev_t = t;
        }
        if (ok && prev_t >= 0) epilogue(i - 1, prev_t);
    }

    // ---- teardown (also after an abort: every role has left its loop)
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

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
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

// Row-major 2D view of the grid; one box is a 32-row slab of an input tile
// (in_w columns, in_w*4-byte TMA rows).
bool encode_tile_map_2d(CUtensorMap* map, const float* base, int ny, int nx, int in_w) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    cuuint64_t strides[1] = {(cuuint64_t)nx * 4};
    cuuint32_t box[2] = {(cuuint32_t)in_w, (cuuint32_t)kSlabRows};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Round to TF32 on the host (nearest, ties to even); finite inputs.
float tf32_round(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    u += 0xFFFu + ((u >> 13) & 1u);
    u &= ~0x1FFFu;
    float y;
    memcpy(&y, &u, 4);
    return y;
}

struct MxState {
    unsigned int* err_host = nullptr;  // host-mapped error word
    unsigned int* err_dev = nullptr;
    int num_sms = 0;
    int nblk = 2;
    uint32_t bop_bytes = 0;
};

}  // namespace

bool mx_supported(const MxRequest& q, std::string* why) {
    if (q.f64) {
        if (why) *why = "FP64 storage runs on the CUDA-core kernel (no FP64 tensor-core path on this GPU)";
        return false;
    }
    if (q.ndim != 2) {
        if (why) *why = "3D matrixized kernel not built";
        return false;
    }
    if (q.prec != STENCIL_PREC_TF32 && q.prec != STENCIL_PREC_TF32X3) {
        if (why) *why = "only TF32 and TF32X3 outer products are built for 2D";
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
    p->nb = kNb;
    const int W = 2 * q.r + 1;
    const int L = W;            // every row a of C^g is one line along the contiguous axis
    const int N = L * kNb;
    // B operand, N x K, K-major core matrices: [part][kchunk][n = a*16 + q][4];
    // entry (n, k) = H_a[k][q] = C^g[a][k - q - (kPad - r)] (banded, Eq. (co)).
    const size_t part_floats = (size_t)kKChunks * N * 4;
    std::vector<float> ops(2 * part_floats, 0.0f);
    for (int a = 0; a < L; ++a) {
        std::vector<double> band((size_t)kK * kNb);
        band_operand(q.r, q.cg + a * W, kNb, kPad, band.data());
        for (int k = 0; k < kK; ++k)
            for (int qq = 0; qq < kNb; ++qq) {
                const float h = (float)band[(size_t)k * kNb + qq];
                const float hi = tf32_round(h);
                const size_t off = (size_t)(k / 4) * N * 4 + (size_t)(a * kNb + qq) * 4 + (k % 4);
                ops[off] = hi;
                ops[part_floats + off] = tf32_round(h - hi);
            }
    }
    p->n_lines = L;
    p->n_scalar = 0;
    p->operand_bytes = ops.size() * sizeof(float);
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
    // Two 16-column blocks per tile while both TMEM stages of A (2 x 2 x in_w
    // columns) and both accumulator sets (2 x nblk x N) fit the 512 columns.
    st->nblk = (2 * 2 * (2 * kNb + 2 * kPad) + 2 * 2 * N <= kTmemCols) ? 2 : 1;
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
    const size_t smem = smem_bytes_2d(st->nblk * kNb + 2 * kPad, st->bop_bytes);
    e = cudaFuncSetAttribute(mx2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        mx_plan_free(p);
        if (why) *why = std::string("shared memory: ") + cudaGetErrorString(e);
        return STENCIL_ECUDA;
    }
    return STENCIL_OK;
}

void mx_plan_free(MxPlan* p) {
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
    const MxState* st = (const MxState*)p.tmap_storage;
    return st && st->err_host ? *(volatile unsigned int*)st->err_host : 0u;
}

cudaError_t mx_sweep(const MxPlan& p, const void* src, void* dst, int tb, cudaStream_t s) {
    if (tb != 1) return cudaErrorInvalidValue;
    if (((uintptr_t)src & 15u) || ((uintptr_t)dst & 15u)) return cudaErrorMisalignedAddress;
    const MxState* st = (const MxState*)p.tmap_storage;
    const int ny = (int)p.n[0], nx = (int)p.n[1];
    MxArgs2D a;
    memset(&a, 0, sizeof(a));
    a.out = (float*)dst;
    a.in = (const float*)src;
    a.bops = (const float*)p.d_operands;
    a.err = st->err_dev;
    a.ny = ny;
    a.nx = nx;
    a.r = p.r;
    a.bc = p.bc;
    a.nlines = p.n_lines;
    a.nprod = (p.prec == STENCIL_PREC_TF32X3) ? 3 : 1;
    a.nblk = st->nblk;
    a.in_w = st->nblk * kNb + 2 * kPad;
    a.rows_out = kSlabRows - 2 * p.r;
    a.tiles_x = (nx + a.nblk * kNb - 1) / (a.nblk * kNb);
    const int tile_rows = kMathWarps * a.rows_out;
    a.tiles_total = a.tiles_x * ((ny + tile_rows - 1) / tile_rows);
    a.bop_bytes = st->bop_bytes;
    alignas(64) CUtensorMap map;
    if (!encode_tile_map_2d(&map, (const float*)src, ny, nx, a.in_w)) return cudaErrorInvalidValue;
    const int grid = a.tiles_total < st->num_sms ? a.tiles_total : st->num_sms;
    mx2d_kernel<<<grid, kThreads, smem_bytes_2d(a.in_w, a.bop_bytes), s>>>(map, a);
    return cudaGetLastError();
}

}  // namespace stx
