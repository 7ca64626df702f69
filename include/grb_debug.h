/* grb_debug.h -- entry points of the bounds-checked build of the library.
 *
 * libgrb_checked.so is the same library compiled with -DGRB_CHECK_BOUNDS;
 * the release library libgrb.so exports none of the calls below.  The paper
 * has no counterpart: this is a debugging aid.  In the checked build
 *   - a matrix's structure (row_ptr starts at 0, ends at nnz, never
 *     decreases; every column index in [0, ncols)) is validated on the
 *     device before the first kernel that walks it (the row-gather plan,
 *     the column counts, the degree-ordered copy, the general mxv), and the
 *     host reads the verdict before anything indexes with it;
 *   - the iterated kernels (the fused row-gather / PageRank kernels, the
 *     batched personalised PageRank tiles, the general mxv) test every
 *     column index they gather with against the vector's extent; a bad one
 *     is replaced by 0 and the first failure is recorded in the context's
 *     device status words.
 * A failure surfaces as GRB_INDEX_OUT_OF_BOUNDS at the next call that reads
 * the status (a wait, the end of a device loop, grb_ppr_status, the
 * graph-batch run); grb_error names the offending index.  No device assert
 * or trap is used: the context stays usable.  Results of a clean run are
 * bit-identical to the release build's.
 */
#ifndef GRB_DEBUG_H
#define GRB_DEBUG_H

#include "grb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Validate a CSR structure given in HOST arrays (row_ptr: nrows + 1
 * entries, col_idx: nnz entries; both only read, caller-owned) on the
 * device with the structure check the library runs before a matrix's first
 * use.  Returns GRB_SUCCESS (*what = 0), or GRB_INDEX_OUT_OF_BOUNDS with
 * *what = 1 and *value = a column index outside [0, ncols), or *what = 2 and
 * *value = a row i whose row_ptr[i] is out of order (row_ptr[i+1] <
 * row_ptr[i]) or outside [0, nnz] (or row_ptr[0] != 0, row_ptr[nrows] !=
 * nnz).  With several failures, which one is reported is unspecified.
 * GRB_NULL_POINTER for a null argument, GRB_INVALID_VALUE for sizes above
 * INT32_MAX.  Synchronises the context's stream. */
grb_info grb_debug_check_csr(grb_context ctx, const int32_t* row_ptr, const int32_t* col_idx, uint64_t nrows,
                             uint64_t ncols, uint64_t nnz, int32_t* what, int64_t* value);

/* Overwrite column index k (< nvals, else GRB_INVALID_INDEX) of A's own
 * column array with col, without any check -- a stand-in for memory
 * corruption after the structure was validated, so that a test can see the
 * in-kernel checks catch it.  The degree-ordered copy of A, if the device
 * loops made one, is not touched.  Synchronises the context's stream. */
grb_info grb_debug_set_col(grb_matrix A, uint64_t k, int32_t col);

#ifdef __cplusplus
}
#endif

#endif /* GRB_DEBUG_H */
