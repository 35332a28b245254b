// Host-side plan of a streamed operator apply (pure C++, no CUDA): how the
// dense rows of every block are cut into work units of `rows` consecutive
// rows x one column piece, where each unit's rows start in the dense layout
// and in the tiled copy, and the tiled row pitch.  The streaming kernels
// (stream.cuh, stream_tc.cuh) read these tables; build_stream_units uploads
// them.
#pragma once

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#if defined(__CUDACC__)
#define MTF_HD __host__ __device__
#else
#define MTF_HD
#endif

namespace mtf {

// row pitch (bytes) of a unit in the tiled copy of a streamed operator with
// eb-byte entries: 4-byte entries (the tensor-core stream) in whole 8-entry
// chunks, padded to 16 bytes past a 128-byte multiple so that the rows an
// ldmatrix phase reads fall in distinct shared-memory banks; others in
// 16-byte words
MTF_HD inline int st_tile_pitch(int eb, int len) {
  if (eb == 4) return ((len + 7) / 8 * 32 + 127) / 128 * 128 + 16;
  return (len * eb + 15) / 16 * 16;
}

struct StreamBlock {
  int N = 0;               // rows (and columns) of the block
  int64_t row_off = 0;     // first global row of the block
  int64_t dof_off = 0;     // first unknown of the block (its D slot)
  int64_t entry_off = 0;   // first entry of the block in the dense layout
  int64_t ld = 0;          // entries between consecutive rows
};

struct StreamPlan {
  // unit record: {N, global row of the first row, dof_off + first column,
  // len | piece << 12 | rows << 24}
  std::vector<int32_t> rec;    // 4 per unit
  std::vector<int64_t> src;    // dense entry offset of the unit's first row piece
  std::vector<int64_t> toff;   // byte offset of the unit in the tiled copy
  int32_t pmax = 1;            // most pieces of any row
  int64_t tiled_bytes = 0;
  int64_t n_units() const { return int64_t(src.size()); }
};

// Every row of block i is cut into P_i = ceil(N_i / piece_len) pieces of
// near-equal length (rounded up to whole 16-byte words), every piece into
// units of `rows` rows.  Returns an empty string, or what is wrong.
inline std::string plan_stream_units(const std::vector<StreamBlock>& blocks, int rows, int piece_len, int eb,
                                     StreamPlan& out) {
  if (eb != 4 && eb != 8 && eb != 16) return "stream entries are 4, 8 or 16 bytes";
  if (rows < 1 || rows > 64) return "rows per stream unit out of range";
  const int q = 16 / eb;  // entries per 16 bytes
  out = StreamPlan{};
  for (const StreamBlock& b : blocks) {
    const int N = b.N;
    const int P = std::max(1, (N + piece_len - 1) / piece_len);
    const int ps = ((N + P - 1) / P + q - 1) / q * q;
    if (ps > piece_len || P >= 4096 || N >= (1 << 30)) return "stream piece longer than a slot";
    if ((b.ld * eb) % 16 != 0 || (b.entry_off * eb) % 16 != 0 || b.ld < N)
      return "stream operator rows are not 16-byte aligned";
    out.pmax = std::max(out.pmax, P);
    for (int p = 0; p < P; ++p) {
      const int c = p * ps, len = std::min(ps, N - c);
      const int clen = (len + q - 1) / q * q;  // entries the copy moves
      if (len <= 0 || len >= 4096 || c + clen > b.ld) return "stream piece out of its row";
      for (int r0 = 0; r0 < N; r0 += rows) {
        const int nr = std::min(rows, N - r0);
        out.rec.push_back(N);
        out.rec.push_back(int32_t(b.row_off + r0));
        out.rec.push_back(int32_t(b.dof_off + c));
        out.rec.push_back(len | (p << 12) | (nr << 24));
        out.src.push_back(b.entry_off + int64_t(r0) * b.ld + c);
        out.toff.push_back(out.tiled_bytes);
        out.tiled_bytes += int64_t(nr) * st_tile_pitch(eb, len);
      }
    }
  }
  if (out.n_units() >= (int64_t(1) << 31)) return "mesh too large for the streaming tables";
  return std::string();
}

}  // namespace mtf
