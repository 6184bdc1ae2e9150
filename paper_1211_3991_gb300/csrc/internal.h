// Internal definitions shared by the host-side translation units of libxyl.
#pragma once

#include <stdarg.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/xyl.h"

namespace xyl {

// Record a failure message (thread local) and return its code.
int fail(int code, const char *fmt, ...);
void clear_error();

}  // namespace xyl

// A graph: creation-order links, lattice coordinates and the colour-sorted CSR.
struct xyl_graph {
    int32_t n = 0;
    int32_t L = 0;          // period of the Fourier phases
    int32_t z = 0;          // fixed degree (0 when built from an edge list)
    int32_t n_colors = 0;
    int32_t max_deg = 0;
    int32_t restarts = 0;
    int64_t n_edges = 0;
    std::vector<int32_t> ei, ej;      // links, creation order, original ids
    std::vector<int32_t> xy;          // 2n coordinates, original ids
    std::vector<int32_t> perm;        // colour-sorted id -> original id
    std::vector<int32_t> row_ptr;     // n + 1
    std::vector<int32_t> col;         // colour-sorted neighbour ids, ascending per row
    std::vector<int32_t> color_ptr;   // n_colors + 1
    std::vector<int32_t> color;       // colour of each original id
    std::vector<int8_t> jlink;        // coupling of each link (creation order), empty = all +1
    std::vector<int8_t> jcsr;         // coupling of each CSR entry (aligned with col), empty = all +1
    std::vector<double> field;        // field_dim x n field components per original id, empty = no field
    int32_t field_dim = 0;            // 2: XY fields (xyl_graph_set_fields), 3: O(3) fields (xyl_graph_set_fields3)
};
