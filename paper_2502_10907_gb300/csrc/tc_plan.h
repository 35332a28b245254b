// Plan of the tensor-core block matvec (mv_tc.cu), pure host C++ so that it
// can be tested on its own.
//
// Formulation.  For block i with dense complex T_i, K_i (N_i x N_i) and the
// inputs u_D, u_N of every right-hand side c, the products T u and K u are
// one real matrix product each: a row of T stored as interleaved (re, im)
// pairs is a real row of length 2 N_i, and a complex input v becomes two real
// columns of the same length,
//   form 0: (v_re, -v_im) per entry -> Re(T v),   form 1: (v_im, v_re) -> Im(T v).
// Column 4 c + 2 t + f of the B operand holds form f of u_t (t = 0: D slot,
// t = 1: N slot) of right-hand side c; NB = 4 nc rounded up to 16, 32, 64 or
// 128 columns (up to 32 right-hand sides per pass).  Both operands are FP16 after a power-of-two scaling (per block
// for T and K, per right-hand side for the inputs) and are split into an FP16
// value and the FP16 rounding of its remainder (hi + lo, about 22 significant
// bits); a product is hi*hi + hi*lo + lo*hi with FP32 accumulation.
//
// Layout.  A tile is (block i, row tile mt of 128 rows, chunk kc of 32
// complex columns = 64 FP16 per row): four parts T hi, T lo, K hi, K lo of
// 128 rows x 64 FP16 (128 bytes per row), 64 KB, tiles of a block in
// (mt, kc) order.  An input chunk is (block i, kc): two parts (hi, lo) of NB
// columns x 64 FP16.  Rows and columns past N_i are zero.  A work unit is
// (block, mt, a range of chunks); the units of (i, mt) are consecutive and
// their per-row partial sums add up to the row's products.  Units are handed
// to the persistent CTAs by longest-processing-time-first scheduling.
#pragma once

#include <algorithm>
#include <cstdint>
#include <queue>
#include <string>
#include <utility>
#include <vector>

namespace mtf {

constexpr int kTcRows = 128;  // rows per tile (M of the MMA)
constexpr int kTcCols = 32;   // complex columns per chunk (64 FP16, 128 bytes)
constexpr int kTcParts = 4;   // T hi, T lo, K hi, K lo
constexpr int64_t kTcPartHalves = int64_t(kTcRows) * 64;
constexpr int64_t kTcTileHalves = kTcParts * kTcPartHalves;

// columns of the B operand for nc (<= 32) right-hand sides: 4 nc rounded up
// to one of the kernel's widths 16, 32, 64, 128
inline int tc_nb(int nc) { return nc <= 4 ? 16 : nc <= 8 ? 32 : nc <= 16 ? 64 : 128; }

// half index of (tile, part, row, e) in tiles of `parts` parts of 128 rows
// x 64 FP16 (constexpr: usable in device code)
constexpr int64_t tc_tile_index(int64_t tile, int parts, int part, int row, int e) {
  return ((tile * parts + part) * kTcRows + row) * 64 + e;
}
// the matvec's operator tiles (4 parts: T hi, T lo, K hi, K lo)
constexpr int64_t tc_a_index(int64_t tile, int part, int row, int e) {
  return tc_tile_index(tile, kTcParts, part, row, e);
}
// half index of (chunk, part 0 hi / 1 lo, column, e) in the input chunks
constexpr int64_t tc_b_index(int64_t chunk, int part, int col, int e, int nb) {
  return ((chunk * 2 + part) * nb + col) * 64 + e;
}

// Tiled FP16 hi / lo copies of a Krylov basis (2-part tiles), the layouts of
// the tensor-core Gram-Schmidt projections (arnoldi_tc.cu), for basis vector
// qq and entry k:
//  - dots copy: tile (qq / 128) nkc + k / 32, row qq % 128, halves 2 (k % 32) + {0, 1};
//  - update copy: tile (k / 128) nbc + qq / 32, row k % 128, halves 2 (qq % 32) + {0, 1};
// with nkc = ldn / 32 entry chunks and nbc = ceil(nvec / 32) basis chunks.
// Returned as the half index of the real part (the imaginary part follows).
constexpr int64_t tca_dots_half(int64_t qq, int64_t k, int64_t nkc, int part) {
  return tc_tile_index((qq / kTcRows) * nkc + k / kTcCols, 2, part, int(qq % kTcRows), int(2 * (k % kTcCols)));
}
constexpr int64_t tca_upd_half(int64_t qq, int64_t k, int64_t nbc, int part) {
  return tc_tile_index((k / kTcRows) * nbc + qq / 32, 2, part, int(k % kTcRows), int(2 * (qq % 32)));
}
// halves of the two copies for nvec basis vectors of padded length ldn
constexpr int64_t tca_dots_halves(int64_t nvec, int64_t ldn) {
  return ((nvec + kTcRows - 1) / kTcRows) * (ldn / kTcCols) * 2 * kTcRows * 64;
}
constexpr int64_t tca_upd_halves(int64_t nvec, int64_t ldn) {
  return ((ldn + kTcRows - 1) / kTcRows) * ((nvec + 31) / 32) * 2 * kTcRows * 64;
}

struct TcBlock {
  int N = 0, n_mt = 0, n_kc = 0, pieces = 1, piece_len = 1;
  int64_t tile_base = 0, chunk_base = 0;
  int unit_base = 0;
};

struct TcUnit {
  int blk, mt, kc0, kc1;
};

struct TcPlan {
  std::vector<TcBlock> blocks;
  std::vector<TcUnit> units;
  std::vector<int> sched, sched_off;  // units of CTA b: sched[sched_off[b] .. sched_off[b+1])
  int64_t n_tiles = 0, n_chunks = 0;
  int64_t max_load = 0, total_load = 0;  // chunks, busiest CTA and all
};

// Pieces of at most piece_len chunks per (block, row tile), piece_len chosen
// so that there are at least `waves` units per CTA on average (but no piece
// shorter than min_len chunks; 0 selects the defaults below); LPT schedule
// over n_cta CTAs.  A chunk covers cols_per_chunk columns of the operator:
// 32 complex columns (64 FP16) for the complex operators, 64 for a real one.
inline std::string plan_tc(const std::vector<int>& Ns, int n_cta, TcPlan& p, int waves = 0, int min_len = 0,
                           int cols_per_chunk = kTcCols) {
  if (n_cta < 1) return "plan_tc: no CTAs";
  if (cols_per_chunk != kTcCols && cols_per_chunk != 2 * kTcCols) return "plan_tc: 32 or 64 columns per chunk";
  p = TcPlan{};
  p.blocks.resize(Ns.size());
  int64_t total_chunks = 0, n_tiles_rows = 0;
  for (size_t i = 0; i < Ns.size(); ++i) {
    TcBlock& b = p.blocks[i];
    if (Ns[i] <= 0) return "plan_tc: empty block";
    b.N = Ns[i];
    b.n_mt = (b.N + kTcRows - 1) / kTcRows;
    b.n_kc = (b.N + cols_per_chunk - 1) / cols_per_chunk;
    total_chunks += int64_t(b.n_mt) * b.n_kc;
    n_tiles_rows += b.n_mt;
  }
  // defaults: long pieces (few row pieces for the combine to add) when every
  // CTA has many chunks, short ones (balance) when it has few
  const bool big = total_chunks >= int64_t(64) * n_cta;
  if (waves <= 0) waves = big ? 4 : 8;
  if (min_len <= 0) min_len = big ? 8 : 2;
  // longest piece that still gives `waves` units per CTA
  int64_t target = std::max<int64_t>(int64_t(min_len), total_chunks / std::max<int64_t>(1, int64_t(waves) * n_cta));
  int64_t tile = 0, chunk = 0;
  int unit = 0;
  for (auto& b : p.blocks) {
    b.pieces = int((b.n_kc + target - 1) / target);
    b.piece_len = (b.n_kc + b.pieces - 1) / b.pieces;
    b.pieces = (b.n_kc + b.piece_len - 1) / b.piece_len;
    b.tile_base = tile;
    b.chunk_base = chunk;
    b.unit_base = unit;
    tile += int64_t(b.n_mt) * b.n_kc;
    chunk += b.n_kc;
    for (int mt = 0; mt < b.n_mt; ++mt)
      for (int q = 0; q < b.pieces; ++q) {
        const int k0 = q * b.piece_len, k1 = std::min(b.n_kc, k0 + b.piece_len);
        p.units.push_back(TcUnit{int(&b - p.blocks.data()), mt, k0, k1});
        ++unit;
      }
  }
  p.n_tiles = tile;
  p.n_chunks = chunk;
  // LPT: longest units first, each to the least-loaded CTA (ties: lowest id)
  std::vector<int> order(p.units.size());
  for (size_t u = 0; u < order.size(); ++u) order[u] = int(u);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (p.units[a].kc1 - p.units[a].kc0) > (p.units[b].kc1 - p.units[b].kc0);
  });
  using Item = std::pair<int64_t, int>;
  std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
  for (int b = 0; b < n_cta; ++b) pq.push({0, b});
  std::vector<std::vector<int>> per(static_cast<size_t>(n_cta));
  for (int u : order) {
    Item it = pq.top();
    pq.pop();
    per[size_t(it.second)].push_back(u);
    it.first += p.units[u].kc1 - p.units[u].kc0;
    p.max_load = std::max(p.max_load, it.first);
    pq.push(it);
  }
  p.total_load = total_chunks;
  p.sched_off.assign(size_t(n_cta) + 1, 0);
  for (int b = 0; b < n_cta; ++b) {
    std::sort(per[size_t(b)].begin(), per[size_t(b)].end());
    p.sched_off[size_t(b) + 1] = p.sched_off[size_t(b)] + int(per[size_t(b)].size());
    p.sched.insert(p.sched.end(), per[size_t(b)].begin(), per[size_t(b)].end());
  }
  (void)n_tiles_rows;
  return "";
}

// Tensor-core formation of the block-OSRC operators T~_i = W_i diag(f_i) W_i^T
// (osrc_form_tc.cu).  W_i is real (N_i x N_i, rows = RWG dofs r, columns =
// modes j) and f_i complex, so with
//   A[r][j] = W(r, j),   B[2 c + t][j] = f_j^(t) W(c, j)   (t = 0: Re, 1: Im)
// the product D = A B^T gives D[r][2 c + t] = (T~_i)^(t)(r, c): the interleaved
// complex rows of T~ directly.  A tile is (block, row tile mt of 128 dofs,
// chunk kc of 64 modes), two parts (hi, lo) of 128 rows x 64 FP16; a B chunk
// is (block, column tile nt of 64 dofs = 128 B rows, chunk kc), two parts of
// 128 rows x 64 FP16.  T~ is symmetric, so only the units (mt, nt) whose
// tile holds an entry with c >= r are formed: a unit writes its entries with
// c >= r in place and those with c > r transposed, so every entry of T~ is
// written exactly once.
constexpr int kTtCols = 64;  // complex output columns per unit (128 B rows)

struct TtBlock {
  int N = 0, n_mt = 0, n_nt = 0, n_kc = 0;
  int64_t a_base = 0, b_base = 0;  // first A tile, first B chunk
};

struct TtUnit {
  int blk, mt, nt;
};

struct TtPlan {
  std::vector<TtBlock> blocks;
  std::vector<TtUnit> units;  // longest blocks first (round-robin over the CTAs)
  int64_t n_a = 0, n_b = 0;   // A tiles, B chunks
};

// does the 128 x 64 output tile (mt, nt) hold an entry with c >= r?
constexpr bool tt_upper(int mt, int nt) { return int64_t(nt) * kTtCols + kTtCols - 1 >= int64_t(mt) * kTcRows; }

inline std::string plan_tt(const std::vector<int>& Ns, TtPlan& p) {
  p = TtPlan{};
  p.blocks.resize(Ns.size());
  int64_t a = 0, b = 0;
  for (size_t i = 0; i < Ns.size(); ++i) {
    TtBlock& q = p.blocks[i];
    if (Ns[i] <= 0) return "plan_tt: empty block";
    q.N = Ns[i];
    q.n_mt = (q.N + kTcRows - 1) / kTcRows;
    q.n_nt = (q.N + kTtCols - 1) / kTtCols;
    q.n_kc = (q.N + 63) / 64;
    q.a_base = a;
    q.b_base = b;
    a += int64_t(q.n_mt) * q.n_kc;
    b += int64_t(q.n_nt) * q.n_kc;
  }
  p.n_a = a;
  p.n_b = b;
  std::vector<int> order(Ns.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = int(i);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return Ns[size_t(x)] > Ns[size_t(y)]; });
  for (int i : order) {
    const TtBlock& q = p.blocks[size_t(i)];
    for (int mt = 0; mt < q.n_mt; ++mt)
      for (int nt = 0; nt < q.n_nt; ++nt)
        if (tt_upper(mt, nt)) p.units.push_back(TtUnit{i, mt, nt});
  }
  return "";
}

}  // namespace mtf
