// Host checks of the streamed-operator plan (stream_plan.h): every dense
// entry of every block belongs to exactly one unit, every bulk copy starts
// and ends on 16-byte boundaries inside its row, and the tiled copy is the
// units' rows back to back at the documented pitch.  Exit 0 and "ok" on
// success.
#include <cstdio>
#include <vector>

#include "stream_plan.h"

using namespace mtf;

static int fails = 0;
#define CHECK(c)                                                        \
  do {                                                                  \
    if (!(c)) {                                                         \
      std::printf("FAIL line %d: %s\n", __LINE__, #c);                  \
      ++fails;                                                          \
    }                                                                   \
  } while (0)

static void run(const std::vector<int>& Ns, int eb, int rows, int piece_len) {
  const int q = 16 / eb;
  std::vector<StreamBlock> bl;
  int64_t row = 0, dof = 0, ent = 0;
  for (int N : Ns) {
    StreamBlock b;
    b.N = N;
    b.row_off = row;
    b.dof_off = dof;
    b.entry_off = ent;
    b.ld = eb == 16 ? N : (eb == 8 ? N + (N & 1) : (N + 3) / 4 * 4);  // the kernels' row strides
    bl.push_back(b);
    row += N;
    dof += 2 * N;
    ent += int64_t(N) * b.ld;
  }
  StreamPlan pl;
  CHECK(plan_stream_units(bl, rows, piece_len, eb, pl).empty());
  // coverage: count how often each (row, column) entry is streamed
  std::vector<int> hits(size_t(ent), 0);
  int64_t expect_off = 0;
  for (int64_t u = 0; u < pl.n_units(); ++u) {
    const int N = pl.rec[4 * u], grow = pl.rec[4 * u + 1], gcol = pl.rec[4 * u + 2], w = pl.rec[4 * u + 3];
    const int len = w & 0xfff, piece = (w >> 12) & 0xfff, nr = (w >> 24) & 0xff;
    int i = 0;
    while (!(grow >= bl[i].row_off && grow < bl[i].row_off + bl[i].N)) ++i;
    const StreamBlock& b = bl[i];
    CHECK(N == b.N && nr >= 1 && nr <= rows && len >= 1 && len <= piece_len && piece < pl.pmax);
    const int r0 = int(grow - b.row_off), c = int(gcol - b.dof_off);
    CHECK(r0 % rows == 0 && r0 + nr <= N && c >= 0 && c + len <= N);
    CHECK(pl.src[u] == b.entry_off + int64_t(r0) * b.ld + c);
    CHECK((pl.src[u] * eb) % 16 == 0 && (b.ld * eb) % 16 == 0);          // every row copy 16-byte aligned
    CHECK(c + (len + q - 1) / q * q <= b.ld);                             // and inside its row
    const int pitch = st_tile_pitch(eb, len);
    CHECK(pitch % 16 == 0 && pitch >= len * eb);
    if (eb == 4) CHECK(pitch % 128 == 16 && pitch >= (len + 7) / 8 * 32);  // bank-conflict-free, whole chunks
    CHECK(pl.toff[u] == expect_off);                                      // units back to back
    expect_off += int64_t(nr) * pitch;
    for (int r = 0; r < nr; ++r)
      for (int e = 0; e < len; ++e) ++hits[size_t(b.entry_off + int64_t(r0 + r) * b.ld + c + e)];
  }
  CHECK(pl.tiled_bytes == expect_off);
  for (const StreamBlock& b : bl)
    for (int r = 0; r < b.N; ++r)
      for (int e = 0; e < b.ld; ++e) CHECK(hits[size_t(b.entry_off + int64_t(r) * b.ld + e)] == (e < b.N ? 1 : 0));
}

int main() {
  // the three stream kinds with their unit rows and piece lengths: {T, K}
  // (16 B, 256 entries), FP32 T~ (8 B, 512), FP16 T~ (4 B, 640)
  const std::vector<std::vector<int>> meshes = {{2178, 2178, 2178}, {7200, 18, 18, 450}, {567}, {1, 2, 3, 4, 5}, {641}};
  for (const auto& Ns : meshes) {
    run(Ns, 16, 16, 256);
    run(Ns, 8, 16, 512);
    run(Ns, 4, 16, 640);
  }
  StreamPlan pl;
  CHECK(!plan_stream_units({}, 0, 256, 16, pl).empty());   // rows out of range
  CHECK(!plan_stream_units({}, 16, 256, 12, pl).empty());  // entry size
  if (fails) return 1;
  std::printf("ok\n");
  return 0;
}
