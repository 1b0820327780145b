// Plan layer: problem validation and the coefficient-line algebra of Sec. 3
// (scatter matrix, coefficient lines, banded line operands).  Host only.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

namespace stx {

// One coefficient line: 2r+1 gather-orientation weights along one axis at a
// fixed offset in the other axes.  `axis` is the axis the line runs along
// (ndim-1 = contiguous).  `fixed` holds the offsets (0..2r) of the other axes
// in axis order, with the line's own axis entry unused.
struct CoefLine {
    int axis;
    int fixed[3];
    std::vector<double> w;  // 2r+1 weights; w[t] multiplies the input at offset t - r
    int first_nz() const;
    int last_nz() const;    // -1 when the line is empty
};

// Scatter-mode coefficient tensor C^s = J C^g J (Eq. (stencil-2d9p-gm2sm)):
// every axis reversed.  Dense, (2r+1)^ndim, C order.
std::vector<double> scatter_tensor(int ndim, int r, const double* cg);

// Lines of a cover option (0 parallel, 1 orthogonal, 2 hybrid) over C^g.
// `line_axis_parallel` is the axis the parallel lines run along.  Every
// nonzero coefficient lands on exactly one line (the centre goes to the
// line along the contiguous axis).  Returns false when the option does not
// apply (message in *why).
bool cover_lines(int ndim, int r, bool star, const double* cg, int option, int line_axis_parallel,
                 std::vector<CoefLine>* lines, std::string* why);

// Outer products one line costs per n-wide output block: n + span - 1, where
// span = last_nz - first_nz + 1 (Sec. 3.4: a full line costs 2r + n, a line
// with one weight costs n).  0 for an empty line.
int64_t line_outer_products(const CoefLine& l, int n);

// Banded operand of a line: K x n, K = n + 2*pad, row-major,
// band[k*n+q] = w[k - q - (pad - r)] inside the band, else 0.
void band_operand(int r, const double* w, int n, int pad, double* band);

}  // namespace stx
