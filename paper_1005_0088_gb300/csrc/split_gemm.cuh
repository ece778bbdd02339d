// Split-precision (emulated FP64) complex GEMM on the tcgen05 tensor cores.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "plan.hpp"

namespace ndsi {

// Tile of the split GEMM: 128 output rows x NC complex output columns.  Default: one TMEM
// accumulator per slice-product scale t+u (S of them, S x 2NC <= 512 columns: NC = 40 for up to
// six slices, 32 for seven), filled by one wide MMA per A digit.  Optional: NC = 64 with four
// accumulators (t+u = 2, 3, 4 exact, the rest in a tail) or NC = 48 with five (t+u = 2..5 exact).
constexpr int kSplitBM = 128;
constexpr int kSplitBNc = 64;      // complex columns per tile, four-band variant
constexpr int kSplitBNc5 = 48;     // complex columns per tile, five-band variant
constexpr int kSplitBNcX = 40;     // complex columns per tile, one accumulator per scale (S <= 6)
constexpr int kSplitBNcX7 = 32;    // the same for seven slices
// Complex columns per tile of a plan: bands 4 or 5 select the tail variants, 0 one accumulator
// per scale.
constexpr int split_nc(int slices, int bands) {
    return bands == 4 ? kSplitBNc : bands == 5 ? kSplitBNc5 : (slices >= 7 ? kSplitBNcX7 : kSplitBNcX);
}
constexpr int kSplitSliceRows = 32;  // operand rows per slicing block (two-pass slicer)
constexpr int kSplitSlice1Smem = 72 * 1024;       // one-pass slicer budget, 4..32 rows per block
constexpr int kSplitSlice1SmemWide = 200 * 1024;  // budget for very long rows, 1 or 2 rows per block
// Stacked K per pipeline stage: 32 BF16 (64-byte rows, 64-byte swizzle, two K16 MMA steps per
// digit).  16 (32-byte rows, 32-byte swizzle) fits five stages at six slices instead of two, but
// its half-size row requests loaded L1 and L2 far more and the 3D metallic sweep ran 9% slower.
#ifdef NDSI_SPLIT_KB
constexpr int kSplitKB = NDSI_SPLIT_KB;
#else
constexpr int kSplitKB = 32;
#endif
static_assert(kSplitKB == 16 || kSplitKB == 32, "stage K must be 16 or 32");
constexpr int kSplitChunkKB = 256 / kSplitKB;   // stages per exact chunk (256 stacked-K elements)
constexpr int kSplitMaxSlices = 7;
// Bytes of one operand's slices a tile group may keep in L2 while the other operand streams
// (a third of GB300's 126 MB L2), and the tiles the persistent GEMM runs at one time (one CTA on
// each of GB300's 152 SMs).
constexpr double kSplitL2Share = 40.0 * 1024 * 1024;
constexpr int kSplitConcurrentTiles = 152;
// Default of ndsi_options.split_far_ratio: density-sweep poles with z_p >= 32 z_1 use one slice
// fewer (32^2 ~ 2^10 covers the 2^8 larger product error of the shorter expansion).
constexpr double kSplitFarRatio = 32.0;

// Where an item's slices and exponents live inside one pole's block of the step buffers.
struct SplitItem {
    int64_t rowA, rowB;     // first slice row of the item (A: S*Mpad rows, B: S*2*Npad rows)
    int64_t erowA, erowB;   // first exponent of the item
    int32_t Mpad, Npad;     // Mpad multiple of 128 rows, Npad multiple of nc complex columns
    int32_t Kpad, pad;      // multiple of kSplitKB (complex K); stacked K is 2*Kpad
};

// Per GEMM launch: sizes of one pole's block in the step buffers, and the split tile range.
struct SplitStep {
    int64_t rowsA, rowsB, erowsA, erowsB;  // per pole
    int32_t Kcols;                         // row length of the slice buffers (2*max Kpad)
    int32_t nc;                            // complex columns per output tile (64, 48, 40 or 32)
    int32_t slice_rows;                    // operand rows per slicing block
    int32_t slice_ldt;                     // one-pass slicing: shared-memory row stride (0: two passes)
    int32_t pad;
    int64_t tfirst, tcount;                // tiles in the split tile list
    int64_t sa_first, sa_count;            // slicing blocks of A (rows of op(A)) in the block list
    int64_t sb_first, sb_count;            // slicing blocks of B (columns of op(B))
};

// A slicing block: item (relative to the launch) and its first row (A) or complex column (B).
struct SliceBlock {
    int32_t item, r0;
};

// Build the split metadata of every GEMM launch (called by the analysis in split mode).
// bands[li]: accumulator layout of launch li (0 one per scale, 4 or 5 with a tail).
void build_split_schedule(const Plan& P, int slices, const std::vector<int8_t>& bands,
                          std::vector<SplitItem>& items, std::vector<SplitStep>& steps,
                          std::vector<GemmTile>& tiles, std::vector<SliceBlock>& blocks);

struct SplitBuffers {
    uint16_t* sliceA = nullptr;   // bf16 bit patterns
    uint16_t* sliceB = nullptr;
    int32_t* expA = nullptr;
    int32_t* expB = nullptr;
    size_t capA = 0, capB = 0, capEA = 0, capEB = 0;  // elements
    std::vector<CUtensorMap> tmA, tmB;                // one per split step (for np_cap poles)
    int32_t np = 0;
};

cudaError_t split_init();
// Allocate the slice buffers for np poles and encode the tensor maps of every step.
cudaError_t split_alloc(SplitBuffers& B, const std::vector<SplitStep>& steps, int slices, int np);
void split_free(SplitBuffers& B);

// One GEMM launch of the schedule in split precision: slice A and B (split_slice_step), then the
// tensor-core product and FP64 epilogue (split_mma_step).
cudaError_t split_slice_step(const Launch& l, const GemmItem* items_dev, const SplitItem* sitems_dev,
                             const SliceBlock* blocks_dev, const SplitStep& step, const SplitBuffers& B,
                             int slices, const double2* Abuf, int64_t sA, const double2* Bbuf, int64_t sB,
                             int np, cudaStream_t st);
cudaError_t split_mma_step(const Launch& l, int step_index, const GemmItem* items_dev,
                           const SplitItem* sitems_dev, const GemmTile* stiles_dev, const SplitStep& step,
                           const SplitBuffers& B, int slices, double2* Cbuf, int64_t sC, int np, int* status,
                           cudaStream_t st);
// Tensor-core flops one pole of the step issues (tiles x 128 x 128 x 2Kpad x pairs x 2).
double split_executed_flops(const Plan& P, const SplitStep& step, const std::vector<SplitItem>& items,
                            const std::vector<GemmTile>& tiles, const Launch& l, int slices);

}  // namespace ndsi
