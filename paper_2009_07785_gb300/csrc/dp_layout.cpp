// One-time host preprocessing of a constraint matrix (the "blocking of the
// matrix precomputed on the CPU" that Sec. 4.3 of arXiv 2009.07785 excludes
// from timing): CSR validation, row chunking, length sorting and the
// slot-major slice image described in dp_internal.h.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "dp_launch.h"
#include "../../include/domprop.h"

namespace dp {

namespace {

// A coefficient outside [2^-120, 2^120] keeps its row out of the binary32
// screen (the screen's bit-level |a| bound assumes a normal binary32 range).
bool coef_screenable(double a) {
  double x = std::fabs(a);
  return x >= 0x1p-120 && x <= 0x1p120;
}

struct Chunk {
  int32_t row;
  int64_t begin;  // CSR offset of the chunk's first nonzero
  int32_t len;
  int32_t flags;  // kExactFlag
  int32_t sidx;   // split-row index or -1
};

}  // namespace

namespace {
// Side class of a row for the ordering within one chunk length: rows whose
// sides have the same finiteness share warps, so a warp whose rows all have
// an infinite side skips that side's activity.  0: both sides finite,
// 1: only rhs finite, 2: only lhs finite, 3: neither.  Without hints every
// row is class 0.
int side_class(const double *lhs, const double *rhs, int32_t i) {
  if (!lhs || !rhs) return 0;
  const double thr = 1e20;
  const bool fl = std::fabs(lhs[i]) < thr, fr = std::fabs(rhs[i]) < thr;
  return fl ? (fr ? 0 : 2) : (fr ? 1 : 3);
}
}  // namespace

namespace {
// Checks a host CSR matrix: offsets from 0 to nnz, non-decreasing; columns
// in range; finite nonzero coefficients.
int validate_csr(int32_t m, int32_t n, int64_t nnz, const int64_t *row_ptr,
                 const int32_t *col_idx, const double *val) {
  if (m < 0 || n < 0 || nnz < 0 || nnz >= (int64_t(1) << 31)) return DP_ERR_INVALID_ARG;
  if (m > 0 && !row_ptr) return DP_ERR_INVALID_ARG;
  if (nnz > 0 && (!col_idx || !val)) return DP_ERR_INVALID_ARG;
  if (m > 0) {
    if (row_ptr[0] != 0 || row_ptr[m] != nnz) return DP_ERR_BAD_CSR;
    for (int32_t i = 0; i < m; ++i)
      if (row_ptr[i + 1] < row_ptr[i]) return DP_ERR_BAD_CSR;
  } else if (nnz != 0) {
    return DP_ERR_BAD_CSR;
  }
  for (int64_t k = 0; k < nnz; ++k) {
    if (col_idx[k] < 0 || col_idx[k] >= n) return DP_ERR_BAD_CSR;
    double a = val[k];
    if (!std::isfinite(a) || a == 0.0) return DP_ERR_BAD_CSR;
  }
  return DP_OK;
}
}  // namespace

int build_layout(int32_t m, int32_t n, int64_t nnz, const int64_t *row_ptr,
                 const int32_t *col_idx, const double *val, int32_t chunk,
                 const double *lhs_hint, const double *rhs_hint, HostLayout &out) {
  if (chunk == 0) chunk = 256;
  if (chunk < 8 || chunk > 4096) return DP_ERR_INVALID_ARG;
  int rc = validate_csr(m, n, nnz, row_ptr, col_idx, val);
  if (rc) return rc;

  try {
    out = HostLayout();
    out.m = m;
    out.n = n;
    out.nnz = nnz;
    std::vector<int32_t> rowflag(m > 0 ? m : 1, 0);
    for (int32_t i = 0; i < m; ++i)
      for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
        if (!coef_screenable(val[k])) { rowflag[i] = kExactFlag; break; }

    // pieces of the split rows, generated row by row (sorted below)
    std::vector<Chunk> chunks;
    chunks.reserve((size_t)m + (size_t)(nnz / chunk) + 1);
    int32_t nsplit = 0;
    for (int32_t i = 0; i < m; ++i) {
      int64_t len = row_ptr[i + 1] - row_ptr[i];
      if (len <= chunk) continue;
      out.split_row.push_back(i);
      out.split_cbeg.push_back((int32_t)chunks.size());
      for (int64_t b = 0; b < len; b += chunk) {
        int64_t e = b + chunk < len ? b + chunk : len;
        chunks.push_back({i, row_ptr[i] + b, (int32_t)(e - b), rowflag[i], nsplit});
      }
      ++nsplit;
    }
    out.split_cbeg.push_back((int32_t)chunks.size());
    out.nsplit_rows = nsplit;
    // sort the split chunks by length too (full chunks, then remainders,
    // longest first) so that lanes of a slice do equal work; split_cidx maps
    // each split row's pieces to their slots
    {
      const size_t ns = chunks.size();
      auto key2 = [&](const Chunk &ch) {
        return (size_t)(chunk - ch.len) * 4 + (size_t)side_class(lhs_hint, rhs_hint, ch.row);
      };
      std::vector<size_t> cnt2(((size_t)chunk + 2) * 4, 0);
      for (const Chunk &ch : chunks) cnt2[key2(ch)]++;
      std::vector<size_t> at2(cnt2.size(), 0);
      for (size_t b = 1; b < at2.size(); ++b) at2[b] = at2[b - 1] + cnt2[b - 1];
      std::vector<Chunk> sorted(ns);
      out.split_cidx.assign(ns, 0);
      for (size_t q = 0; q < ns; ++q) {
        size_t slot = at2[key2(chunks[q])]++;
        sorted[slot] = chunks[q];
        out.split_cidx[q] = (int32_t)slot;
      }
      chunks.swap(sorted);
    }
    // pad the split region to whole slices so no slice mixes both kinds
    while (chunks.size() % kSliceW) chunks.push_back({-1, 0, 0, 0, -1});
    const size_t nsplit_chunks = chunks.size();

    // single-chunk rows by length, longest first, then by side class
    // (counting sort, stable)
    auto key1 = [&](int32_t i, int64_t len) {
      return (size_t)(chunk - len) * 4 + (size_t)side_class(lhs_hint, rhs_hint, i);
    };
    std::vector<int64_t> cnt(((size_t)chunk + 2) * 4, 0);
    for (int32_t i = 0; i < m; ++i) {
      int64_t len = row_ptr[i + 1] - row_ptr[i];
      if (len <= chunk) cnt[key1(i, len)]++;
    }
    std::vector<int64_t> pos(cnt.size(), 0);
    for (size_t b = 1; b < pos.size(); ++b) pos[b] = pos[b - 1] + cnt[b - 1];
    size_t nsingle = (size_t)(pos.back() + cnt.back());
    chunks.resize(nsplit_chunks + nsingle);
    for (int32_t i = 0; i < m; ++i) {
      int64_t len = row_ptr[i + 1] - row_ptr[i];
      if (len > chunk) continue;
      size_t at = nsplit_chunks + (size_t)pos[key1(i, len)]++;
      chunks[at] = {i, row_ptr[i], (int32_t)len, rowflag[i], -1};
    }
    while (chunks.size() % kSliceW) chunks.push_back({-1, 0, 0, 0, -1});

    const size_t nslots = chunks.size();
    // queue entries pack the chunk slot in 30 bits and the element offset
    // in 32 bits
    if (nslots >= (size_t(1) << 30)) return DP_ERR_INVALID_ARG;
    out.nslices = (int32_t)(nslots / kSliceW);
    out.nslices_split = (int32_t)(nsplit_chunks / kSliceW);
    out.slice_off.resize(out.nslices);
    out.slice_len.resize(out.nslices);
    int64_t total = 0;
    for (int32_t s = 0; s < out.nslices; ++s) {
      int32_t L = 0;
      for (int t = 0; t < kSliceW; ++t) {
        int32_t l = chunks[(size_t)s * kSliceW + t].len;
        if (l > L) L = l;
      }
      out.slice_off[s] = total;
      out.slice_len[s] = L;
      total += (int64_t)L * kSliceW;
    }
    // candidate work lists address elements with 32-bit offsets
    if (total >= (int64_t(1) << 32)) return DP_ERR_INVALID_ARG;
    out.val.assign((size_t)total, 0.0);
    out.col.assign((size_t)total, 0);
    // lossless int8 copy of the values when every coefficient is a small
    // integer (the round kernels then stream 1 byte per value, not 8)
    bool small = true;
    for (int64_t k = 0; k < nnz && small; ++k) {
      const double a = val[k];
      small = a == std::nearbyint(a) && std::fabs(a) <= 127.0;
    }
    if (small) out.val8.assign((size_t)total, 0);
    out.chunk_row.resize(nslots);
    out.chunk_len.resize(nslots);
    out.chunk_sidx.assign(nsplit_chunks, -1);
    for (size_t c = 0; c < nslots; ++c) {
      const Chunk &ch = chunks[c];
      out.chunk_row[c] = ch.row;
      out.chunk_len[c] = ch.len | ch.flags;
      if (c < nsplit_chunks) out.chunk_sidx[c] = ch.sidx;
      int64_t base = out.slice_off[c / kSliceW] + (int64_t)(c % kSliceW);
      for (int32_t k = 0; k < ch.len; ++k) {
        out.val[(size_t)(base + (int64_t)k * kSliceW)] = val[ch.begin + k];
        out.col[(size_t)(base + (int64_t)k * kSliceW)] = col_idx[ch.begin + k];
        if (small) out.val8[(size_t)(base + (int64_t)k * kSliceW)] = (int8_t)val[ch.begin + k];
      }
    }
  } catch (const std::bad_alloc &) {
    return DP_ERR_OOM;
  }
  return DP_OK;
}

// Merge-path layout (dp_internal.h): rows in side-class order (stable), the
// merged sequence of row ends and nonzeros cut into segments of `ipt`
// items, the first row of each segment, and the split rows with their
// pieces.  In the merged sequence the first nonzero of row p (side-class
// order) is item p + ptr[p] and its row end is item p + ptr[p+1]; a row is
// split when these fall in different segments ta < tb, and its pieces are
// the carry of ta, the carries of the segments in between (which hold
// nothing but nonzeros of the row) and the head of tb.
int build_merge_layout(int32_t m, int32_t n, int64_t nnz, const int64_t *row_ptr,
                       const int32_t *col_idx, const double *val, int32_t ipt,
                       const double *lhs_hint, const double *rhs_hint, HostLayout &out) {
  if (ipt < 4 || ipt > 4096) return DP_ERR_INVALID_ARG;
  int rc = validate_csr(m, n, nnz, row_ptr, col_idx, val);
  if (rc) return rc;
  const int64_t total = (int64_t)m + nnz;
  const int64_t nseg = (total + ipt - 1) / ipt;
  // piece indices (2 per segment) and row offsets are 32-bit
  if (2 * nseg >= (int64_t(1) << 31)) return DP_ERR_INVALID_ARG;
  try {
    out = HostLayout();
    out.m = m;
    out.n = n;
    out.nnz = nnz;
    out.layout = kLayoutMerge;
    out.mp_ipt = ipt;
    out.mp_nseg = (int32_t)nseg;
    out.nslices = (m + kSliceW - 1) / kSliceW;
    // queue entries pack the row in 30 bits
    if ((int64_t)out.nslices * kSliceW >= (int64_t(1) << 30)) return DP_ERR_INVALID_ARG;
    // rows by side class, stable (no hints: CSR order)
    std::vector<int32_t> perm((size_t)m);
    {
      int64_t cnt[5] = {0, 0, 0, 0, 0};
      for (int32_t i = 0; i < m; ++i) cnt[side_class(lhs_hint, rhs_hint, i) + 1]++;
      for (int c = 1; c < 5; ++c) cnt[c] += cnt[c - 1];
      for (int32_t i = 0; i < m; ++i) perm[(size_t)cnt[side_class(lhs_hint, rhs_hint, i)]++] = i;
    }
    const size_t nslots = (size_t)out.nslices * kSliceW;
    out.chunk_row.assign(nslots > 0 ? nslots : 0, -1);
    out.chunk_len.assign(nslots > 0 ? nslots : 0, 0);
    out.mp_ptr.assign((size_t)m + 1, 0);
    out.val.resize((size_t)nnz);
    out.col.resize((size_t)nnz);
    int64_t at = 0;
    for (int32_t p = 0; p < m; ++p) {
      const int32_t i = perm[(size_t)p];
      int32_t flag = 0;
      for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k, ++at) {
        out.val[(size_t)at] = val[k];
        out.col[(size_t)at] = col_idx[k];
        if (!coef_screenable(val[k])) flag = kExactFlag;
      }
      out.mp_ptr[(size_t)p + 1] = (int32_t)at;
      out.chunk_row[(size_t)p] = i;
      out.chunk_len[(size_t)p] = (int32_t)(row_ptr[i + 1] - row_ptr[i]) | flag;
    }
    // rows whose end precedes each segment's first item (a walk of the
    // merged sequence: a nonzero k of row p comes before p's row end)
    out.mp_srow.assign((size_t)nseg + 1, m);
    {
      int32_t p = 0;
      int64_t k = 0;
      for (int64_t t = 0; t <= nseg; ++t) {
        const int64_t d = t * ipt < total ? t * ipt : total;
        while (p + k < d) {
          if (p < m && k < out.mp_ptr[(size_t)p + 1]) ++k;
          else ++p;
        }
        out.mp_srow[(size_t)t] = p;
      }
    }
    // split rows and their pieces
    out.split_cbeg.push_back(0);
    for (int32_t p = 0; p < m; ++p) {
      const int64_t ta = ((int64_t)p + out.mp_ptr[(size_t)p]) / ipt;
      const int64_t tb = ((int64_t)p + out.mp_ptr[(size_t)p + 1]) / ipt;
      if (ta == tb) continue;
      out.split_row.push_back(p);
      for (int64_t t = ta; t < tb; ++t) out.split_cidx.push_back((int32_t)(2 * t + 1));
      out.split_cidx.push_back((int32_t)(2 * tb));
      out.split_cbeg.push_back((int32_t)out.split_cidx.size());
    }
    out.nsplit_rows = (int32_t)out.split_row.size();
    // long rows: their screen re-read is cut into pieces, one warp each
    out.chunk_sidx.assign(nslots, -1);
    for (int32_t p = 0; p < m; ++p) {
      const int32_t b = out.mp_ptr[(size_t)p], len = out.mp_ptr[(size_t)p + 1] - b;
      if (len <= kMpLaneRow) continue;
      out.chunk_sidx[(size_t)p] = out.mp_nlong;
      for (int32_t o = 0; o < len; o += kMpPiece)
        out.mp_piece.push_back(make_int4(p, out.mp_nlong, b + o, len - o < kMpPiece ? len - o : kMpPiece));
      ++out.mp_nlong;
    }
  } catch (const std::bad_alloc &) {
    return DP_ERR_OOM;
  }
  return DP_OK;
}

}  // namespace dp
