// Host-only operations on RACE plans beyond their construction: the reverse
// Cuthill-McKee relabelling applied before it, and the inverse of the
// canonical export image.  Implemented in race_builder.cpp.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "race_internal.h"

namespace race {

// Reverse Cuthill-McKee order (order[new] = old) of the symmetric graph of a
// canonical upper CRS: components in the order of their lowest vertex, each
// from a pseudo-peripheral vertex of it, breadth first with the neighbours
// newly reached from a vertex taken by increasing degree (lowest index on
// ties); the whole sequence reversed.
std::vector<int32_t> rcm_order(int32_t n, const int32_t* row_ptr, const int32_t* col);

// Inverse of export_plan for a matrix of n rows: every field is checked
// (sizes, permutation, phase offsets, leaves covering each row exactly
// once, the tree's shape); false with the reason in `why` on any mismatch.
bool import_plan(const void* buf, size_t size, int32_t n, Plan& out, std::string& why);

}  // namespace race
