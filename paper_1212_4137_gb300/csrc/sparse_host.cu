// sparse_host.cu -- host-side preparation of a sparse A given in compressed sparse rows: input
// checks, the canonical layouts by rows and by columns, and the SpMM work items.
//   sp_canonical  checks the row offsets, column indices and values; builds A by columns (A^T by
//                 rows) with a counting sort over the rows in order (each column's rows come out
//                 ascending, a repeated (i, j) entry adjacent), sums the repeats in input order,
//                 and builds A by rows back from it (columns ascending, none repeated);
//   sp_plan       cuts the rows into work items of at most kSpItemNnz entries: runs of up to
//                 kSpItemRows consecutive rows, or equal segments of a longer row (whose partial
//                 sums a fix-up adds in segment order).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "spca_internal.cuh"

namespace spca {

namespace {
// CSR of the transpose of (ptr, col, val) (rows x cols), rows visited in order
void transpose_csr(int64_t rows, int64_t cols, const int64_t *ptr, const int32_t *col, const float *val,
                   HostCsr *T) {
  const int64_t nnz = ptr[rows];
  T->rows = cols;
  T->cols = rows;
  T->ptr.assign((size_t)cols + 1, 0);
  for (int64_t k = 0; k < nnz; ++k) ++T->ptr[(size_t)col[k] + 1];
  for (int64_t j = 0; j < cols; ++j) T->ptr[(size_t)j + 1] += T->ptr[(size_t)j];
  T->col.resize((size_t)nnz);
  T->val.resize((size_t)nnz);
  std::vector<int64_t> pos(T->ptr.begin(), T->ptr.end() - 1);
  for (int64_t i = 0; i < rows; ++i)
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
      const int64_t q = pos[(size_t)col[k]]++;
      T->col[(size_t)q] = (int)i;
      T->val[(size_t)q] = val[k];
    }
}
}  // namespace

const char *sp_canonical(int64_t n, int64_t p, int64_t nnz, const int64_t *ptr, const int32_t *col,
                         const float *val, HostCsr *A, HostCsr *AT) {
  if (ptr[0] != 0 || ptr[n] != nnz) return "row_ptr[0] must be 0 and row_ptr[n] must be nnz";
  for (int64_t i = 0; i < n; ++i)
    if (ptr[i + 1] < ptr[i]) return "row_ptr must be non-decreasing";
  for (int64_t k = 0; k < nnz; ++k) {
    if (col[k] < 0 || (int64_t)col[k] >= p) return "a column index is out of range";
    if (!std::isfinite(val[k])) return "A has a non-finite entry";
  }
  // by columns, repeats adjacent, then summed in place
  HostCsr C;
  transpose_csr(n, p, ptr, col, val, &C);
  int64_t w = 0;
  for (int64_t j = 0; j < p; ++j) {
    const int64_t b = C.ptr[(size_t)j], e = C.ptr[(size_t)j + 1];
    C.ptr[(size_t)j] = w;
    for (int64_t k = b; k < e; ++k) {
      if (k > b && C.col[(size_t)k] == C.col[(size_t)k - 1]) {
        C.val[(size_t)w - 1] += C.val[(size_t)k];
      } else {
        C.col[(size_t)w] = C.col[(size_t)k];
        C.val[(size_t)w] = C.val[(size_t)k];
        ++w;
      }
    }
  }
  C.ptr[(size_t)p] = w;
  C.col.resize((size_t)w);
  C.val.resize((size_t)w);
  for (int64_t k = 0; k < w; ++k)
    if (!std::isfinite(C.val[(size_t)k])) return "a sum of repeated entries is not finite";
  // by rows from the canonical columns: columns ascending within each row
  transpose_csr(p, n, C.ptr.data(), C.col.data(), C.val.data(), A);
  *AT = std::move(C);
  return nullptr;
}

void sp_plan(const std::vector<int64_t> &ptr, std::vector<SpItem> *items, std::vector<SpLong> *longs, int *nseg) {
  const int64_t rows = (int64_t)ptr.size() - 1;
  items->clear();
  longs->clear();
  int seg = 0;
  for (int64_t i = 0; i < rows;) {
    const int64_t len = ptr[(size_t)i + 1] - ptr[(size_t)i];
    if (len > kSpItemNnz) {
      const int64_t parts = (len + kSpItemNnz - 1) / kSpItemNnz;
      const int64_t per = (len + parts - 1) / parts;
      longs->push_back(SpLong{(int)i, seg, (int)parts, 0});
      for (int64_t g = 0; g < parts; ++g) {
        const int64_t b = std::min<int64_t>(ptr[(size_t)i + 1], ptr[(size_t)i] + g * per);
        const int64_t e = std::min<int64_t>(ptr[(size_t)i + 1], b + per);
        items->push_back(SpItem{(int)i, (int)i + 1, seg + (int)g, 0, b, e});
      }
      seg += (int)parts;
      ++i;
      continue;
    }
    int64_t j = i, tot = 0;
    while (j < rows && j - i < kSpItemRows) {
      const int64_t l = ptr[(size_t)j + 1] - ptr[(size_t)j];
      if (l > kSpItemNnz || tot + l > kSpItemNnz) break;
      tot += l;
      ++j;
    }
    items->push_back(SpItem{(int)i, (int)j, -1, 0, ptr[(size_t)i], ptr[(size_t)j]});
    i = j;
  }
  *nseg = seg;
}

}  // namespace spca
