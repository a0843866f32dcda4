// Host building blocks of the incomplete-LU preconditioner of the mechanical block
// (Sec. 3.3.1): the paper replaces A11 = E + C^ep, for preconditioning, by C^ep plus the
// fraction p of the near-field entries of E with the largest magnitude, and applies the
// inverse of that sparse matrix through an incomplete LU factorization.
//
// Rules (the paper names neither the level of fill, nor a tie rule, nor an ordering):
//   * selection: the ceil(p n) entries of largest |v|, ties by (row, column) ascending
//     (a repeated pair by input position);
//   * ILU(0): no fill outside the pattern, no pivoting; row by row, each entry left of
//     the diagonal becomes the multiplier a_rb / u_bb and row b of U, scaled by it, is
//     taken off the entries of row r that are in the pattern (rows b ascending);
//   * leaf colours: greedy in leaf order, the smallest colour none of the already
//     coloured neighbours holds (two leaves are neighbours when the pattern couples
//     them, in either direction);
//   * levels of the triangular solves: a row waits for every row its pattern names
//     below (lower solve) or above (upper solve) the diagonal.
// This file is compiled with floating-point contraction disabled so that the
// factorization is the plain IEEE sequence written here.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.h"
#include "hmat.h"

namespace hm {
namespace {

// rows sorted, columns in range, diagonal present; returns the diagonal position of
// every row
std::vector<int64_t> check_csr(int32_t n, const int64_t* rowptr, const int32_t* col) {
    if (n < 0) fail(HM_EINVAL, "ilu: negative dimension");
    if (n > 0 && (!rowptr || !col)) fail(HM_EINVAL, "ilu: NULL pattern");
    std::vector<int64_t> diag(n, -1);
    if (n > 0 && rowptr[0] != 0) fail(HM_EINVAL, "ilu: the first row pointer must be 0");
    for (int32_t r = 0; r < n; ++r) {
        if (rowptr[r + 1] < rowptr[r]) fail(HM_EINVAL, "ilu: row pointers decrease");
        for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) {
            if (col[q] < 0 || col[q] >= n) fail(HM_EINVAL, "ilu: column out of range");
            if (q > rowptr[r] && col[q] <= col[q - 1]) fail(HM_EINVAL, "ilu: columns not strictly increasing");
            if (col[q] == r) diag[r] = q;
        }
        if (diag[r] < 0) fail(HM_EINVAL, "ilu: the diagonal is not in the pattern");
    }
    return diag;
}

}  // namespace
}  // namespace hm

extern "C" {

hm_status hm_ilu_select(int64_t n, const int32_t* i, const int32_t* j, const double* v, double p,
                        int64_t* idx_out, int64_t* m_out) {
    HM_API_BEGIN
    if (n < 0 || !m_out) hm::fail(HM_EINVAL, "ilu_select: bad size or NULL count");
    if (!(p > 0.0 && p <= 1.0)) hm::fail(HM_EINVAL, "ilu_select: p must lie in (0, 1]");
    if (n > 0 && (!i || !j || !v || !idx_out)) hm::fail(HM_EINVAL, "ilu_select: NULL array");
    for (int64_t q = 0; q < n; ++q)
        if (!std::isfinite(v[q])) hm::fail(HM_ENAN, "ilu_select: NaN or Inf value");
    const int64_t m = (int64_t)std::ceil(p * (double)n);
    std::vector<int64_t> ord(n);
    std::iota(ord.begin(), ord.end(), (int64_t)0);
    auto before = [&](int64_t a, int64_t b) {
        const double fa = std::fabs(v[a]), fb = std::fabs(v[b]);
        if (fa != fb) return fa > fb;
        if (i[a] != i[b]) return i[a] < i[b];
        if (j[a] != j[b]) return j[a] < j[b];
        return a < b;  // a repeated (i, j): input order
    };
    std::partial_sort(ord.begin(), ord.begin() + m, ord.end(), before);
    std::copy(ord.begin(), ord.begin() + m, idx_out);
    *m_out = m;
    HM_API_END
}

hm_status hm_ilu_assemble(int32_t n, int64_t n_entries, int64_t m, const int64_t* idx, const int32_t* i,
                          const int32_t* j, const double* v, const double* d, const int32_t* order,
                          int64_t* rowptr_out, int32_t* col_out, double* val_out, int64_t* nnz_out) {
    HM_API_BEGIN
    if (n < 0 || m < 0 || n_entries < 0) hm::fail(HM_EINVAL, "ilu_assemble: negative size");
    if ((m > 0 && (!idx || !i || !j || !v)) || (n > 0 && (!d || !col_out || !val_out)) || !rowptr_out)
        hm::fail(HM_EINVAL, "ilu_assemble: NULL array");
    // new position of every old row (order: new -> old; NULL: identity)
    std::vector<int32_t> newpos(n);
    if (order) {
        std::vector<char> seen(n, 0);
        for (int32_t q = 0; q < n; ++q) {
            if (order[q] < 0 || order[q] >= n || seen[order[q]]) hm::fail(HM_EINVAL, "ilu_assemble: order is not a permutation");
            seen[order[q]] = 1;
            newpos[order[q]] = q;
        }
    } else {
        std::iota(newpos.begin(), newpos.end(), 0);
    }
    // entries per new row: the selected ones, then the diagonal
    std::vector<std::vector<std::pair<int32_t, double>>> rows(n);
    for (int64_t t = 0; t < m; ++t) {
        const int64_t q = idx[t];
        if (q < 0 || q >= n_entries) hm::fail(HM_EINVAL, "ilu_assemble: entry index outside the entry list");
        if (i[q] < 0 || i[q] >= n || j[q] < 0 || j[q] >= n) hm::fail(HM_EINVAL, "ilu_assemble: entry out of range");
        rows[newpos[i[q]]].push_back({newpos[j[q]], v[q]});
    }
    int64_t nnz = 0;
    rowptr_out[0] = 0;
    for (int32_t r = 0; r < n; ++r) {
        auto& row = rows[r];
        std::sort(row.begin(), row.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        for (size_t q = 1; q < row.size(); ++q)
            if (row[q].first == row[q - 1].first) hm::fail(HM_EINVAL, "ilu_assemble: entry selected twice");
        // -d on the diagonal, which is always in the pattern
        auto it = std::lower_bound(row.begin(), row.end(), r, [](const auto& a, int32_t c) { return a.first < c; });
        const double dr = d[order ? order[r] : r];
        if (it != row.end() && it->first == r)
            it->second = it->second - dr;
        else
            row.insert(it, {r, 0.0 - dr});
        for (const auto& e : row) {
            col_out[nnz] = e.first;
            val_out[nnz] = e.second;
            ++nnz;
        }
        rowptr_out[r + 1] = nnz;
    }
    if (nnz_out) *nnz_out = nnz;
    HM_API_END
}

hm_status hm_ilu0_factor(int32_t n, const int64_t* rowptr, const int32_t* col, double* val) {
    HM_API_BEGIN
    const std::vector<int64_t> diag = hm::check_csr(n, rowptr, col);
    if (n > 0 && !val) hm::fail(HM_EINVAL, "ilu0_factor: NULL values");
    std::vector<int64_t> at(n, -1);  // position of each column in the current row
    for (int32_t r = 0; r < n; ++r) {
        for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) at[col[q]] = q;
        for (int64_t q = rowptr[r]; q < diag[r]; ++q) {
            const int32_t b = col[q];
            const double ub = val[diag[b]];
            if (ub == 0.0) hm::fail(HM_EBREAKDOWN, "ilu0_factor: zero pivot");
            const double l = val[q] / ub;
            val[q] = l;
            for (int64_t t = diag[b] + 1; t < rowptr[b + 1]; ++t) {
                const int64_t pos = at[col[t]];
                if (pos >= 0) val[pos] -= l * val[t];
            }
        }
        for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) at[col[q]] = -1;
    }
    HM_API_END
}

hm_status hm_ilu_levels(int32_t n, const int64_t* rowptr, const int32_t* col, int32_t* lower_out,
                        int32_t* upper_out, int32_t* n_lower_out, int32_t* n_upper_out) {
    HM_API_BEGIN
    const std::vector<int64_t> diag = hm::check_csr(n, rowptr, col);
    std::vector<int32_t> lo(n, 0), up(n, 0);
    int32_t nlo = 0, nup = 0;
    for (int32_t r = 0; r < n; ++r) {
        int32_t l = 0;
        for (int64_t q = rowptr[r]; q < diag[r]; ++q) l = std::max(l, lo[col[q]] + 1);
        lo[r] = l;
        nlo = std::max(nlo, l + 1);
    }
    for (int32_t r = n - 1; r >= 0; --r) {
        int32_t l = 0;
        for (int64_t q = diag[r] + 1; q < rowptr[r + 1]; ++q) l = std::max(l, up[col[q]] + 1);
        up[r] = l;
        nup = std::max(nup, l + 1);
    }
    if (lower_out) std::copy(lo.begin(), lo.end(), lower_out);
    if (upper_out) std::copy(up.begin(), up.end(), upper_out);
    if (n_lower_out) *n_lower_out = nlo;
    if (n_upper_out) *n_upper_out = nup;
    HM_API_END
}

hm_status hm_ilu_leaf_colours(int32_t n, const int64_t* rowptr, const int32_t* col, const int32_t* leaf_of,
                              int32_t n_leaves, int32_t* colour_out, int32_t* n_colours_out) {
    HM_API_BEGIN
    if (n < 0 || n_leaves < 0) hm::fail(HM_EINVAL, "ilu_leaf_colours: negative size");
    if (n > 0 && !leaf_of) hm::fail(HM_EINVAL, "ilu_leaf_colours: NULL array");
    hm::check_csr(n, rowptr, col);
    if (n_leaves > 0 && !colour_out) hm::fail(HM_EINVAL, "ilu_leaf_colours: NULL output");
    for (int32_t r = 0; r < n; ++r)
        if (leaf_of[r] < 0 || leaf_of[r] >= n_leaves) hm::fail(HM_EINVAL, "ilu_leaf_colours: leaf out of range");
    std::vector<std::vector<int32_t>> nbr(n_leaves);
    for (int32_t r = 0; r < n; ++r)
        for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) {
            const int32_t a = leaf_of[r], b = leaf_of[col[q]];
            if (a != b) {
                nbr[a].push_back(b);
                nbr[b].push_back(a);
            }
        }
    std::vector<int32_t> colour(n_leaves, -1);
    int32_t nc = 0;
    std::vector<char> used;
    for (int32_t l = 0; l < n_leaves; ++l) {
        used.assign((size_t)nc + 1, 0);
        for (int32_t m : nbr[l])
            if (colour[m] >= 0) used[colour[m]] = 1;
        int32_t c = 0;
        while (used[c]) ++c;
        colour[l] = c;
        nc = std::max(nc, c + 1);
    }
    if (n_leaves > 0) std::copy(colour.begin(), colour.end(), colour_out);
    if (n_colours_out) *n_colours_out = nc;
    HM_API_END
}

}  // extern "C"
