// Code builders of libbpsf (host only): bivariate bicycle / generalised
// bicycle check matrices (Appendix "Code Construction") and the R-round
// phenomenological detector matrix.
#include <algorithm>
#include <vector>

#include "bpsf.h"
#include "bpsf_api_internal.h"

// Monomial x^a y^b with x = S_l (x) I_m, y = I_l (x) S_m: S_l has its one in
// row r at column (r + 1) mod l, so x^a y^b maps row (r1, r2) = r1*m + r2 to
// column ((r1 + a) mod l) * m + (r2 + b) mod m.  Its transpose maps row
// (r1, r2) to ((r1 - a) mod l) * m + (r2 - b) mod m.
static int mono_col(int r, int a, int b, int l, int m, bool transpose) {
    const int r1 = r / m, r2 = r % m;
    int c1, c2;
    if (!transpose) {
        c1 = ((r1 + a) % l + l) % l;
        c2 = ((r2 + b) % m + m) % m;
    } else {
        c1 = ((r1 - a) % l + l) % l;
        c2 = ((r2 - b) % m + m) % m;
    }
    return c1 * m + c2;
}

extern "C" bpsf_status bpsf_bb_code(int32_t l, int32_t m, int32_t n_a, const int32_t *a_x, const int32_t *a_y,
                                    int32_t n_b, const int32_t *b_x, const int32_t *b_y, int32_t which,
                                    int32_t *ptr_out, int32_t *idx_out, int64_t idx_cap, int64_t *nnz_out) {
    if (l < 1 || m < 1 || (long long)l * m > 32767) return bpsf_fail(BPSF_EINVAL, "l*m must be in 1..32767");
    if (n_a < 0 || n_b < 0 || (n_a && (!a_x || !a_y)) || (n_b && (!b_x || !b_y)))
        return bpsf_fail(BPSF_EINVAL, "bad polynomial terms");
    if (which != 0 && which != 1) return bpsf_fail(BPSF_EINVAL, "which must be 0 (H_X) or 1 (H_Z)");
    if (!ptr_out || !idx_out || !nnz_out) return bpsf_fail(BPSF_EINVAL, "NULL output");
    const int n = l * m;
    // H_X = [A | B];  H_Z = [B^T | A^T].
    const int nl = which == 0 ? n_a : n_b, nr = which == 0 ? n_b : n_a;
    const int32_t *lx = which == 0 ? a_x : b_x, *ly = which == 0 ? a_y : b_y;
    const int32_t *rx = which == 0 ? b_x : a_x, *ry = which == 0 ? b_y : a_y;
    const bool tr = which == 1;
    long long nnz = 0;
    ptr_out[0] = 0;
    std::vector<int> cols;
    for (int r = 0; r < n; ++r) {
        cols.clear();
        for (int t = 0; t < nl; ++t) cols.push_back(mono_col(r, lx[t], ly[t], l, m, tr));
        for (int t = 0; t < nr; ++t) cols.push_back(n + mono_col(r, rx[t], ry[t], l, m, tr));
        std::sort(cols.begin(), cols.end());
        // Repeated monomials cancel modulo 2.
        for (size_t k = 0; k < cols.size();) {
            size_t e = k;
            while (e < cols.size() && cols[e] == cols[k]) ++e;
            if ((e - k) & 1) {
                if (nnz >= idx_cap) return bpsf_fail(BPSF_ENOMEM, "idx_cap too small");
                idx_out[nnz++] = cols[k];
            }
            k = e;
        }
        ptr_out[r + 1] = (int32_t)nnz;
    }
    *nnz_out = nnz;
    return BPSF_OK;
}

extern "C" bpsf_status bpsf_phenom_code(int32_t M0, int32_t N0, const int32_t *ptr0, const int32_t *idx0,
                                        int32_t rounds, int32_t *ptr_out, int32_t *idx_out, int64_t idx_cap,
                                        int64_t *nnz_out) {
    if (M0 < 1 || N0 < 1 || rounds < 1 || !ptr0 || !idx0 || !ptr_out || !idx_out || !nnz_out)
        return bpsf_fail(BPSF_EINVAL, "bad arguments");
    const long long R = rounds;
    long long nnz = 0;
    ptr_out[0] = 0;
    for (long long t = 0; t < R; ++t)
        for (int j = 0; j < M0; ++j) {
            // Data errors of round t seen through H0 ...
            for (int k = ptr0[j]; k < ptr0[j + 1]; ++k) {
                if (idx0[k] < 0 || idx0[k] >= N0) return bpsf_fail(BPSF_EINVAL, "index out of range");
                if (nnz >= idx_cap) return bpsf_fail(BPSF_ENOMEM, "idx_cap too small");
                idx_out[nnz++] = (int32_t)(t * N0 + idx0[k]);
            }
            // ... then the measurement errors of rounds t-1 and t on check j.
            const long long mbase = R * N0;
            if (t > 0) {
                if (nnz >= idx_cap) return bpsf_fail(BPSF_ENOMEM, "idx_cap too small");
                idx_out[nnz++] = (int32_t)(mbase + (t - 1) * M0 + j);
            }
            if (nnz >= idx_cap) return bpsf_fail(BPSF_ENOMEM, "idx_cap too small");
            idx_out[nnz++] = (int32_t)(mbase + t * M0 + j);
            ptr_out[t * M0 + j + 1] = (int32_t)nnz;
        }
    *nnz_out = nnz;
    return BPSF_OK;
}
