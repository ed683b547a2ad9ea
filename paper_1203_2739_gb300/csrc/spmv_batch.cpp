// Batched plans: many independent matrices in one plan, so that one exec is
// one launch over all of them.  The batch is the block-diagonal matrix
// diag(A_1, ..., A_B); its x_hat and y_hat are the per-matrix vectors back to
// back.  A split batch merges the k-th parts of all matrices into its k-th
// part, so the batch is itself a nonzero-disjoint split (Sec. 4) of the
// block-diagonal matrix.
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "spmv_internal.h"

using namespace spmv;

extern "C" spmv_status spmv_plan_create_batched(int32_t count, const spmv_csr *A,
                                                const spmv_perm *perms,
                                                const spmv_splits *splits,
                                                const spmv_opts *opts, spmv_plan **out)
{
    clear_error();
    if (!out) {
        set_error("out is NULL");
        return SPMV_E_INVALID;
    }
    *out = nullptr;
    if (count < 1 || !A) {
        set_error("count=%d: a batch needs at least one matrix", count);
        return SPMV_E_INVALID;
    }
    try {
        int64_t M = 0, N = 0, NNZ = 0;
        for (int32_t b = 0; b < count; ++b) {
            spmv_status st = validate_csr(&A[b]);
            if (st != SPMV_OK) {
                const std::string why = spmv_last_error();
                set_error("matrix %d: %s", b, why.c_str());
                return st;
            }
            M += A[b].m;
            N += A[b].n;
            NNZ += A[b].nnz;
        }
        if (M >= INT32_MAX || N >= INT32_MAX || NNZ >= INT32_MAX) {
            set_error("the batch has %lld rows, %lld columns, %lld nonzeros: each must fit int32",
                      (long long)M, (long long)N, (long long)NNZ);
            return SPMV_E_UNSUPPORTED;
        }
        int32_t form = SPMV_NATURAL, K = 1;
        if (splits) {
            form = splits[0].form;
            K = splits[0].K;
            for (int32_t b = 0; b < count; ++b) {
                if (splits[b].form != form || (form == SPMV_SPLIT && splits[b].K != K)) {
                    set_error("matrix %d: every matrix of a batch needs the same form (and K)", b);
                    return SPMV_E_INVALID;
                }
            }
            if (form != SPMV_NATURAL && form != SPMV_SPLIT) {
                set_error("batched plans take the natural or the split form (SB/DB borders "
                          "of different matrices cannot share one border)");
                return SPMV_E_UNSUPPORTED;
            }
            if (form == SPMV_SPLIT && K < 1) {
                set_error("K=%d must be >= 1", K);
                return SPMV_E_INVALID;
            }
        }
        std::vector<int32_t> rp((size_t)M + 1, 0), ci((size_t)NNZ);
        std::vector<double> val((size_t)NNZ);
        std::vector<int32_t> rperm, cperm, nzp;
        bool any_perm = false;
        for (int32_t b = 0; b < count && perms; ++b)
            any_perm = any_perm || perms[b].row_perm || perms[b].col_perm;
        if (any_perm) {
            rperm.resize((size_t)M);
            cperm.resize((size_t)N);
        }
        if (form == SPMV_SPLIT) nzp.resize((size_t)NNZ);
        int64_t r0 = 0, c0 = 0, e0 = 0;
        for (int32_t b = 0; b < count; ++b) {
            const spmv_csr &a = A[b];
            for (int32_t i = 0; i < a.m; ++i) rp[r0 + i + 1] = (int32_t)(e0 + a.rowptr[i + 1]);
            for (int64_t p = 0; p < a.nnz; ++p) {
                ci[e0 + p] = (int32_t)(c0 + a.colidx[p]);
                val[e0 + p] = a.vals[p];
            }
            if (form == SPMV_SPLIT) {
                if (!splits[b].nz_part && a.nnz > 0) {
                    set_error("matrix %d: split form needs nz_part", b);
                    return SPMV_E_INVALID;
                }
                for (int64_t p = 0; p < a.nnz; ++p) {
                    const int32_t k = splits[b].nz_part[p];
                    if (k < 0 || k >= K) {
                        set_error("matrix %d: nz_part[%lld]=%d outside [0, %d)", b, (long long)p,
                                  k, K);
                        return SPMV_E_INVALID;
                    }
                    nzp[e0 + p] = k;
                }
            }
            if (any_perm) {
                const int32_t *pr = perms[b].row_perm, *pc = perms[b].col_perm;
                for (int32_t i = 0; i < a.m; ++i) {
                    const int32_t v = pr ? pr[i] : i;
                    if (v < 0 || v >= a.m) {
                        set_error("matrix %d: row_perm[%d]=%d out of range", b, i, v);
                        return SPMV_E_STRUCTURE;
                    }
                    rperm[r0 + i] = (int32_t)(r0 + v);
                }
                for (int32_t j = 0; j < a.n; ++j) {
                    const int32_t v = pc ? pc[j] : j;
                    if (v < 0 || v >= a.n) {
                        set_error("matrix %d: col_perm[%d]=%d out of range", b, j, v);
                        return SPMV_E_STRUCTURE;
                    }
                    cperm[c0 + j] = (int32_t)(c0 + v);
                }
            }
            r0 += a.m;
            c0 += a.n;
            e0 += a.nnz;
        }
        spmv_csr big{(int32_t)M, (int32_t)N, NNZ, rp.data(), ci.data(), val.data()};
        spmv_perm bp{any_perm ? rperm.data() : nullptr, any_perm ? cperm.data() : nullptr};
        spmv_splits bs{form, K, nullptr, nullptr, form == SPMV_SPLIT ? nzp.data() : nullptr};
        return spmv_plan_create(&big, any_perm ? &bp : nullptr,
                                form == SPMV_SPLIT ? &bs : nullptr, opts, out);
    } catch (const std::bad_alloc &) {
        set_error("out of host memory");
        return SPMV_E_NOMEM;
    }
}
