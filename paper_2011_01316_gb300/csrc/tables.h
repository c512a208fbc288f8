// Host-side LGL tables (nodes, weights, differentiation matrix).
#pragma once
#include "../../include/expdg.h"

namespace expdg {
// r[p+1], w[p+1], D[(p+1)*(p+1)] row-major (D[i*(p+1)+j] = l_j'(r_i)).
void build_lgl(int p, double* r, double* w, double* D);
}  // namespace expdg
