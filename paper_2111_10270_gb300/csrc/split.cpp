// Long-row splitting (fdog_split_rows): a row sum_{i in I} x_i <= 1 (or = 1)
// over more than max_len variables becomes a chain of short rows joined by
// auxiliary binaries y_1 .. y_{m-1}:
//
//   sum_{P_1} x - y_1 = 0,   y_{j-1} + sum_{P_j} x - y_j = 0,   y_{m-1} + sum_{P_m} x <= 1 (= 1)
//
// Consecutive pieces share one binary variable, so the convex hull of the
// chain, projected onto x, is the convex hull of the original row (two
// 0-1 sets glued along a single binary variable: condition both on its value
// and pair the conditional decompositions).  The Lagrange decomposition over
// the split rows therefore has the same optimal bound, with BDDs of at most
// max_len layers instead of one of |I| layers (the long-row handling the
// paper's conclusion names as future work).
#include <cstdint>
#include <vector>

#include "fdog_internal.h"

namespace {

bool splittable(const int64_t* row_ptr, const int32_t* coef, const int8_t* sense, const int64_t* rhs, int32_t j,
                int32_t max_len) {
    const int64_t len = row_ptr[j + 1] - row_ptr[j];
    if (len <= max_len || rhs[j] != 1 || (sense[j] != FDOG_LE && sense[j] != FDOG_EQ)) return false;
    for (int64_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q)
        if (coef[q] != 1) return false;
    return true;
}

// variables of each piece of a row of `len` entries (first piece max_len - 1,
// middle pieces max_len - 2, the last piece the rest, at most max_len - 1)
std::vector<int64_t> piece_sizes(int64_t len, int32_t max_len) {
    std::vector<int64_t> p;
    int64_t rest = len - (max_len - 1);
    p.push_back(max_len - 1);
    while (rest > max_len - 1) {
        p.push_back(max_len - 2);
        rest -= max_len - 2;
    }
    p.push_back(rest);
    return p;
}

}  // namespace

extern "C" int fdog_split_rows(int32_t n_vars, int32_t n_rows, const int64_t* row_ptr, const int32_t* col,
                               const int32_t* coef, const int8_t* sense, const int64_t* rhs, int32_t max_len,
                               int32_t* out_n_vars, int32_t* out_n_rows, int64_t* out_nnz, int64_t* out_row_ptr,
                               int32_t* out_col, int32_t* out_coef, int8_t* out_sense, int64_t* out_rhs,
                               int32_t* out_row_origin) {
    if (n_vars < 0 || n_rows < 0 || max_len < 3 || !out_n_vars || !out_n_rows || !out_nnz) return FDOG_EINVAL;
    if (n_rows > 0 && (!row_ptr || !sense || !rhs || row_ptr[0] != 0)) return FDOG_EINVAL;
    for (int32_t j = 0; j < n_rows; ++j)
        if (row_ptr[j + 1] < row_ptr[j]) return FDOG_EINVAL;
    if (n_rows > 0 && row_ptr[n_rows] > 0 && (!col || !coef)) return FDOG_EINVAL;
    // sizes: every split row of m pieces adds m - 1 variables, m - 1 rows and 2 (m - 1) entries
    int64_t nv = n_vars, nr = n_rows, nnz = n_rows > 0 ? row_ptr[n_rows] : 0;
    for (int32_t j = 0; j < n_rows; ++j) {
        if (!splittable(row_ptr, coef, sense, rhs, j, max_len)) continue;
        const int64_t m = static_cast<int64_t>(piece_sizes(row_ptr[j + 1] - row_ptr[j], max_len).size());
        nv += m - 1;
        nr += m - 1;
        nnz += 2 * (m - 1);
    }
    if (nv > INT32_MAX || nr > INT32_MAX) return FDOG_EUNSUPPORTED;
    const bool query = !out_row_ptr;
    if (!query && (*out_n_vars < nv || *out_n_rows < nr || *out_nnz < nnz || !out_col || !out_coef || !out_sense ||
                   !out_rhs))
        return FDOG_EINVAL;
    *out_n_vars = static_cast<int32_t>(nv);
    *out_n_rows = static_cast<int32_t>(nr);
    *out_nnz = nnz;
    if (query) return FDOG_OK;

    int32_t y = n_vars;  // next auxiliary variable
    int64_t r = 0, q = 0;
    out_row_ptr[0] = 0;
    auto put = [&](int32_t c, int32_t a) {
        out_col[q] = c;
        out_coef[q] = a;
        ++q;
    };
    auto end_row = [&](int8_t s, int64_t b, int32_t origin) {
        out_sense[r] = s;
        out_rhs[r] = b;
        if (out_row_origin) out_row_origin[r] = origin;
        out_row_ptr[++r] = q;
    };
    for (int32_t j = 0; j < n_rows; ++j) {
        const int64_t b = row_ptr[j], e = row_ptr[j + 1];
        if (!splittable(row_ptr, coef, sense, rhs, j, max_len)) {
            for (int64_t k = b; k < e; ++k) put(col[k], coef[k]);
            end_row(sense[j], rhs[j], j);
            continue;
        }
        const std::vector<int64_t> p = piece_sizes(e - b, max_len);
        int64_t at = b;
        // entries in ascending column order when the row's are (auxiliaries
        // are numbered after every original variable, in creation order)
        for (size_t piece = 0; piece < p.size(); ++piece) {
            for (int64_t k = 0; k < p[piece]; ++k) put(col[at++], 1);
            if (piece > 0) put(y - 1, 1);  // y_{piece}: the sum of the pieces before
            if (piece + 1 < p.size()) {
                put(y++, -1);
                end_row(FDOG_EQ, 0, j);
            } else {
                end_row(sense[j], 1, j);
            }
        }
    }
    return FDOG_OK;
}
