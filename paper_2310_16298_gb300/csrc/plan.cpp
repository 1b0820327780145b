// Plan layer: coefficient-line algebra (Sec. 3.1-3.5 and Sec. 4.1).
#include "plan.h"

#include <cmath>

namespace stx {

int CoefLine::first_nz() const {
    for (size_t t = 0; t < w.size(); ++t)
        if (w[t] != 0.0) return (int)t;
    return -1;
}

int CoefLine::last_nz() const {
    for (int t = (int)w.size() - 1; t >= 0; --t)
        if (w[t] != 0.0) return t;
    return -1;
}

static int64_t lin_index(int ndim, int W, const int* o) {
    int64_t l = 0;
    for (int d = 0; d < ndim; ++d) l = l * W + o[d];
    return l;
}

std::vector<double> scatter_tensor(int ndim, int r, const double* cg) {
    const int W = 2 * r + 1;
    int64_t n = 1;
    for (int d = 0; d < ndim; ++d) n *= W;
    std::vector<double> cs((size_t)n);
    int o[3], ro[3];
    for (int64_t t = 0; t < n; ++t) {
        int64_t rem = t;
        for (int d = ndim - 1; d >= 0; --d) {
            o[d] = (int)(rem % W);
            rem /= W;
            ro[d] = 2 * r - o[d];  // J reverses every axis
        }
        cs[(size_t)t] = cg[lin_index(ndim, W, ro)];
    }
    return cs;
}

// The line along `axis` through the fixed offsets `fx` (entries of other axes).
static CoefLine extract(int ndim, int r, const double* cg, int axis, const int* fx) {
    const int W = 2 * r + 1;
    CoefLine l;
    l.axis = axis;
    for (int d = 0; d < 3; ++d) l.fixed[d] = (d < ndim) ? fx[d] : 0;
    l.w.resize(W);
    int o[3];
    for (int d = 0; d < ndim; ++d) o[d] = fx[d];
    for (int t = 0; t < W; ++t) {
        o[axis] = t;
        l.w[t] = cg[lin_index(ndim, W, o)];
    }
    return l;
}

bool cover_lines(int ndim, int r, bool star, const double* cg, int option, int axis_par,
                 std::vector<CoefLine>* lines, std::string* why) {
    const int W = 2 * r + 1;
    lines->clear();
    if (option == 0) {
        // All lines parallel to axis_par that carry a nonzero weight.
        int fx[3] = {0, 0, 0};
        const int others = ndim - 1;
        int64_t count = 1;
        for (int d = 0; d < others; ++d) count *= W;
        for (int64_t t = 0; t < count; ++t) {
            int64_t rem = t;
            for (int d = ndim - 1; d >= 0; --d) {
                if (d == axis_par) {
                    fx[d] = 0;
                    continue;
                }
                fx[d] = (int)(rem % W);
                rem /= W;
            }
            CoefLine l = extract(ndim, r, cg, axis_par, fx);
            if (l.last_nz() >= 0) lines->push_back(l);
        }
        return true;
    }
    if (!star) {
        if (why) *why = "orthogonal and hybrid covers apply to star stencils only";
        return false;
    }
    const int cont = ndim - 1;
    if (option == 1) {
        for (int axis = 0; axis < ndim; ++axis) {
            int fx[3] = {r, r, r};
            CoefLine l = extract(ndim, r, cg, axis, fx);
            if (axis != cont) l.w[r] = 0.0;  // the centre weight belongs to the contiguous line
            lines->push_back(l);
        }
        return true;
    }
    if (option == 2) {
        if (ndim != 3) {
            if (why) *why = "the hybrid cover is defined for 3D star stencils";
            return false;
        }
        // CLS(i,*,r) for i = 0..2r (lines along axis 1), then CLS(r,r,*).
        for (int i = 0; i < W; ++i) {
            int fx[3] = {i, 0, r};
            CoefLine l = extract(ndim, r, cg, 1, fx);
            if (i == r) l.w[r] = 0.0;
            lines->push_back(l);
        }
        int fx[3] = {r, r, 0};
        lines->push_back(extract(ndim, r, cg, 2, fx));
        return true;
    }
    if (why) *why = "unknown cover option";
    return false;
}

int64_t line_outer_products(const CoefLine& l, int n) {
    const int f = l.first_nz();
    if (f < 0) return 0;
    const int span = l.last_nz() - f + 1;
    return (int64_t)n + span - 1;
}

void band_operand(int r, const double* w, int n, int pad, double* band) {
    const int K = n + 2 * pad;
    const int s = pad - r;
    for (int k = 0; k < K; ++k)
        for (int q = 0; q < n; ++q) {
            const int t = k - q - s;
            band[(size_t)k * n + q] = (t >= 0 && t <= 2 * r) ? w[t] : 0.0;
        }
}

}  // namespace stx
