// Which warps take their transposed products in FP64 and which in
// double-float arithmetic, for a share of fp64_quarters out of every four.
//
// An SM deals its resident warps to its four sub-partitions by warp index
// modulo 4, and every sub-partition issues to its own FP64 unit.  Picking the
// FP64 warps by warp index modulo 4 would put the whole FP64 share on
// fp64_quarters of the four units and leave the others idle.  Instead the
// choice is made per warp-wide group of rows: the group's number (its first
// row divided by the rows a warp takes at once; consecutive for the warps of
// one pass over the grid, strided by the grid's warp count from one pass to
// the next) is hashed to a quarter by multiplicative "Fibonacci" hashing
// (Knuth, TAOCP vol. 3, Sec. 6.4), whose values for evenly spaced keys are
// evenly spread.  Each FP64 unit then carries the same share over the kernel
// and, at any moment, the warps resident on a unit are spread over the four
// quarters.  Warp-uniform whenever `group` is; no register is carried across
// iterations.
#pragma once
#include <cstdint>

__device__ __forceinline__ bool fp64_group(uint32_t group, int fp64_quarters) {
    return ((group * 0x9E3779B9u) >> 30) < static_cast<uint32_t>(fp64_quarters);
}
