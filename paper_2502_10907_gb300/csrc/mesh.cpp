// Skeleton-mesh processing on the host: Algorithm 1 of the paper ("Process
// subdomains and swap normals", Sec. 4.2), the RWG tables of every Gamma_i,
// the singular triangle-pair lists of every block and the sparse structure
// of the transmission Grams (Eq. 18).  Integer bookkeeping only; every
// floating-point quantity of the method is computed by the device kernels,
// except the per-triangle RWG coefficients s l / (2 A) and areas, which are
// uploaded with the geometry.
#include <algorithm>
#include <cmath>
#include <map>
#include <unordered_map>

#include "common.h"

namespace mtf {

static inline int64_t edge_key(int32_t u, int32_t v, int64_t nv) {
  return int64_t(std::min(u, v)) * (nv + 1) + std::max(u, v);
}

mtf_mesh build_mesh(const double* V, int32_t nv, const int32_t* F, int32_t nt, const int32_t* L,
                    int32_t nd) {
  MTF_REQUIRE(V && F && L, MTF_ERR_ARG, "null input array");
  MTF_REQUIRE(nv >= 3 && nt >= 1 && nd >= 2, MTF_ERR_ARG, "need nv >= 3, nt >= 1, n_domains >= 2");
  auto* m = new mtf_mesh_s();
  try {
    m->nv = nv;
    m->nt = nt;
    m->nd = nd;
    m->V.assign(V, V + size_t(nv) * 3);
    m->F.assign(F, F + size_t(nt) * 3);
    m->L.assign(L, L + size_t(nt) * 2);
    for (int32_t t = 0; t < nt; ++t) {
      int32_t a = m->L[2 * t], b = m->L[2 * t + 1];
      MTF_REQUIRE(a >= 0 && b >= 0 && a < nd && b < nd && a != b, MTF_ERR_MESH,
                  "triangle " + std::to_string(t) + " has invalid labels");
      for (int q = 0; q < 3; ++q)
        MTF_REQUIRE(m->F[3 * t + q] >= 0 && m->F[3 * t + q] < nv, MTF_ERR_MESH,
                    "triangle " + std::to_string(t) + " has a vertex id out of range");
      // normal from min(i, j) to max(i, j) (Sec. 3.2): flip if needed
      if (a > b) {
        std::swap(m->L[2 * t], m->L[2 * t + 1]);
        std::swap(m->F[3 * t + 1], m->F[3 * t + 2]);
      }
    }
    // triangles of each interface Gamma_ij (i < j), ascending
    std::map<std::pair<int, int>, std::vector<int32_t>> iface;
    for (int32_t t = 0; t < nt; ++t) iface[{m->L[2 * t], m->L[2 * t + 1]}].push_back(t);
    std::vector<std::vector<int>> Lambda(nd);
    for (auto& kv : iface) {
      Lambda[kv.first.first].push_back(kv.first.second);
      Lambda[kv.first.second].push_back(kv.first.first);
    }
    m->blk.resize(nd);
    int64_t bt = 0, dofo = 0, mato = 0, rowo = 0;
    std::vector<std::unordered_map<int32_t, int32_t>> bt_of(nd);  // skeleton tri -> block-tri
    for (int i = 0; i < nd; ++i) {
      std::sort(Lambda[i].begin(), Lambda[i].end());
      MTF_REQUIRE(!Lambda[i].empty(), MTF_ERR_MESH, "subdomain " + std::to_string(i) + " has no triangles");
      BlockInfo& B = m->blk[i];
      B.bt_off = bt;
      // Algorithm 1: for each j in Lambda_i, swap = sign(j - i), and the
      // triangles of Gamma_ij join RWG_i with that swap.
      for (int j : Lambda[i]) {
        const int swap = j > i ? 1 : -1;
        for (int32_t t : iface[{std::min(i, j), std::max(i, j)}]) {
          bt_of[i][t] = int32_t(bt);
          m->bt_tri.push_back(t);
          m->bt_swap.push_back(int8_t(swap));
          m->bt_blk.push_back(i);
          ++bt;
        }
      }
      B.T = int32_t(bt - B.bt_off);
      // dofs: edges of Gamma_i by increasing (lo, hi) vertex id
      std::vector<int64_t> keys;
      keys.reserve(size_t(B.T) * 3);
      for (int64_t q = B.bt_off; q < bt; ++q) {
        const int32_t* f = &m->F[3 * m->bt_tri[q]];
        for (int a = 0; a < 3; ++a) keys.push_back(edge_key(f[(a + 1) % 3], f[(a + 2) % 3], nv));
      }
      std::vector<int64_t> uk = keys;
      std::sort(uk.begin(), uk.end());
      // closedness: every edge of Gamma_i on exactly two of its triangles
      for (size_t q = 0; q < uk.size();) {
        size_t r = q;
        while (r < uk.size() && uk[r] == uk[q]) ++r;
        MTF_REQUIRE(r - q == 2, MTF_ERR_MESH,
                    "Gamma_" + std::to_string(i) + " is not a closed surface (an edge lies on " +
                        std::to_string(r - q) + " of its triangles)");
        q = r;
      }
      uk.erase(std::unique(uk.begin(), uk.end()), uk.end());
      B.N = int32_t(uk.size());
      for (int64_t q = B.bt_off; q < bt; ++q) {
        const int32_t t = m->bt_tri[q];
        const int32_t* f = &m->F[3 * t];
        const double* p0 = &m->V[3 * f[0]];
        const double* p1 = &m->V[3 * f[1]];
        const double* p2 = &m->V[3 * f[2]];
        double e1[3], e2[3], cr[3];
        for (int c = 0; c < 3; ++c) { e1[c] = p1[c] - p0[c]; e2[c] = p2[c] - p0[c]; }
        cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
        cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
        cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double area = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        MTF_REQUIRE(area > 0, MTF_ERR_MESH, "degenerate triangle " + std::to_string(t));
        m->bt_area.push_back(area);
        for (int a = 0; a < 3; ++a) {
          const int32_t u = f[(a + 1) % 3], w = f[(a + 2) % 3];
          const int64_t key = edge_key(u, w, nv);
          const int32_t d = int32_t(std::lower_bound(uk.begin(), uk.end(), key) - uk.begin());
          m->bt_dof.push_back(d);
          m->bt_vid.push_back(f[a]);
          const double* pu = &m->V[3 * u];
          const double* pw = &m->V[3 * w];
          const double l = std::sqrt((pu[0] - pw[0]) * (pu[0] - pw[0]) + (pu[1] - pw[1]) * (pu[1] - pw[1]) +
                                     (pu[2] - pw[2]) * (pu[2] - pw[2]));
          const int dir = u < w ? 1 : -1;
          m->bt_c.push_back(dir * m->bt_swap[q] * l / (2.0 * area));
        }
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) m->bt_v.push_back(m->V[3 * f[a] + c]);
      }
      // P1 (vertex) tables of Gamma_i: local vertex ids, per-dof (lo, hi) and length
      {
        std::vector<int32_t> verts;
        for (int64_t q = B.bt_off; q < bt; ++q)
          for (int a = 0; a < 3; ++a) verts.push_back(m->F[3 * m->bt_tri[q] + a]);
        std::sort(verts.begin(), verts.end());
        verts.erase(std::unique(verts.begin(), verts.end()), verts.end());
        m->p1_n.push_back(int32_t(verts.size()));
        auto loc = [&](int32_t v) { return int32_t(std::lower_bound(verts.begin(), verts.end(), v) - verts.begin()); };
        for (int64_t q = B.bt_off; q < bt; ++q)
          for (int a = 0; a < 3; ++a) m->bt_lv.push_back(loc(m->F[3 * m->bt_tri[q] + a]));
        for (size_t d = 0; d < uk.size(); ++d) {
          const int32_t lo = int32_t(uk[d] / (int64_t(nv) + 1)), hi = int32_t(uk[d] % (int64_t(nv) + 1));
          m->edge_lohi.push_back(loc(lo));
          m->edge_lohi.push_back(loc(hi));
          const double* pl = &m->V[3 * lo];
          const double* ph = &m->V[3 * hi];
          m->edge_len.push_back(std::sqrt((pl[0] - ph[0]) * (pl[0] - ph[0]) + (pl[1] - ph[1]) * (pl[1] - ph[1]) +
                                          (pl[2] - ph[2]) * (pl[2] - ph[2])));
        }
        m->p1_off_h.push_back(m->p1_nmat);
        m->p1_row_h.push_back(m->p1_nrow);
        m->p1_nmat += int64_t(verts.size()) * int64_t(verts.size());
        m->p1_nrow += int64_t(verts.size());
      }
      B.dof_off = dofo;
      B.mat_off = mato;
      B.row_off = rowo;
      dofo += 2 * int64_t(B.N);
      mato += int64_t(B.N) * B.N;
      rowo += B.N;
    }
    m->n_bt = bt;
    m->n_total = dofo;
    m->n_mat = mato;
    m->n_rows = rowo;

    // ---- singular pairs per block (shared vertices) ------------------------
    for (int i = 0; i < nd; ++i) {
      const BlockInfo& B = m->blk[i];
      std::unordered_map<int32_t, std::vector<int32_t>> v2t;
      for (int64_t q = B.bt_off; q < B.bt_off + B.T; ++q)
        for (int a = 0; a < 3; ++a) v2t[m->F[3 * m->bt_tri[q] + a]].push_back(int32_t(q));
      int64_t cnt[3] = {0, 0, 0};
      for (int64_t q = B.bt_off; q < B.bt_off + B.T; ++q) {
        const int32_t* ft = &m->F[3 * m->bt_tri[q]];
        std::vector<int32_t> cand;
        for (int a = 0; a < 3; ++a)
          for (int32_t s : v2t[ft[a]]) cand.push_back(s);
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        for (int32_t s : cand) {
          const int32_t* fs = &m->F[3 * m->bt_tri[s]];
          int shared = 0;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) shared += ft[a] == fs[b];
          // T and K are symmetric Galerkin forms: an edge- or vertex-adjacent
          // pair is integrated once, with the lower-indexed triangle as the
          // test triangle, and its entries are also added transposed for the
          // swapped pair (the counts below still count ordered pairs)
          if (shared < 3 && s < q) continue;
          int kind, pt[3], ps[3];
          if (shared == 3) {
            kind = 0;
            for (int a = 0; a < 3; ++a) pt[a] = ps[a] = a;
          } else if (shared == 2) {
            kind = 1;
            int sa = -1;
            for (int a = 0; a < 3 && sa < 0; ++a) {
              bool inA = false, inB = false;
              for (int b = 0; b < 3; ++b) {
                inA |= fs[b] == ft[a];
                inB |= fs[b] == ft[(a + 1) % 3];
              }
              if (inA && inB) sa = a;
            }
            pt[0] = sa; pt[1] = (sa + 1) % 3; pt[2] = (sa + 2) % 3;
            for (int b = 0; b < 3; ++b) {
              if (fs[b] == ft[pt[0]]) ps[0] = b;
              else if (fs[b] == ft[pt[1]]) ps[1] = b;
              else ps[2] = b;
            }
          } else {
            kind = 2;
            int sa = 0, sb = 0;
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b)
                if (ft[a] == fs[b]) { sa = a; sb = b; }
            for (int c = 0; c < 3; ++c) { pt[c] = (sa + c) % 3; ps[c] = (sb + c) % 3; }
          }
          cnt[kind] += kind == 0 ? 1 : 2;
          SingPair sp;
          sp.tau = int32_t(q);
          sp.sig = s;
          sp.block = i;
          sp.code = kind | (pt[0] << 2) | (pt[1] << 4) | (pt[2] << 6) | (ps[0] << 8) | (ps[1] << 10) |
                    (ps[2] << 12);
          m->sing.push_back(sp);
        }
      }
      for (int c = 0; c < 3; ++c) m->pair_counts[c] += cnt[c];
      m->pair_counts[3] += int64_t(B.T) * B.T - cnt[0] - cnt[1] - cnt[2];
    }
    // sort singular pairs by kind so that warps of one launch see similar work
    std::stable_sort(m->sing.begin(), m->sing.end(),
                     [](const SingPair& a, const SingPair& b) { return (a.code & 3) < (b.code & 3); });

    // ---- exchange rows (transmission Grams, Eq. 18) ------------------------
    m->dof_bt.assign(size_t(m->n_rows) * 2, -1);
    for (int i = 0; i < nd; ++i) {
      const BlockInfo& B = m->blk[i];
      for (int64_t q = B.bt_off; q < B.bt_off + B.T; ++q)
        for (int a = 0; a < 3; ++a) {
          const int64_t row = B.row_off + m->bt_dof[3 * q + a];
          int32_t* slot = &m->dof_bt[2 * row];
          if (slot[0] < 0) slot[0] = int32_t(3 * q + a);
          else slot[1] = int32_t(3 * q + a);
        }
    }
    m->xent.resize(size_t(m->n_rows) * 6);
    for (int64_t row = 0; row < m->n_rows; ++row)
      for (int e = 0; e < 2; ++e) {
        const int32_t code = m->dof_bt[2 * row + e];
        const int32_t q = code / 3, a = code % 3;
        const int32_t t = m->bt_tri[q];
        const int i = m->bt_blk[q];
        const int j = m->L[2 * t] == i ? m->L[2 * t + 1] : m->L[2 * t];
        const int32_t qj = bt_of[j].at(t);
        for (int b = 0; b < 3; ++b) {
          XEntry& x = m->xent[size_t(row) * 6 + e * 3 + b];
          x.bt_i = q;
          x.bt_j = qj;
          x.col = int32_t(m->blk[j].dof_off + m->bt_dof[3 * qj + b]);
          x.ab = a | (b << 2) | (m->blk[j].N << 4);
        }
      }
    return m;
  } catch (...) {
    delete m;
    throw;
  }
}

void upload_mesh(mtf_mesh m, cudaStream_t s) {
  m->d_bt_v.upload(m->bt_v, s);
  m->d_bt_c.upload(m->bt_c, s);
  m->d_bt_area.upload(m->bt_area, s);
  m->d_bt_dof.upload(m->bt_dof, s);
  m->d_bt_vid.upload(m->bt_vid, s);
  m->d_bt_blk.upload(m->bt_blk, s);
  m->d_bt_swap.upload(m->bt_swap, s);
  m->d_sing.upload(m->sing, s);
  m->d_xent.upload(m->xent, s);
  m->d_dof_bt.upload(m->dof_bt, s);
  m->d_bt_lv.upload(m->bt_lv, s);
  m->d_p1_n.upload(m->p1_n, s);
  m->d_p1_off.upload(m->p1_off_h, s);
  m->d_edge_lohi.upload(m->edge_lohi, s);
  m->d_edge_len.upload(m->edge_len, s);
  std::vector<int64_t> mo, bo, dofo, rowo;
  std::vector<int32_t> N, T, row_blk;
  m->reg_cta_prefix.assign(1, 0);
  for (int i = 0; i < m->nd; ++i) {
    mo.push_back(m->blk[i].mat_off);
    bo.push_back(m->blk[i].bt_off);
    dofo.push_back(m->blk[i].dof_off);
    rowo.push_back(m->blk[i].row_off);
    N.push_back(m->blk[i].N);
    T.push_back(m->blk[i].T);
    const int64_t pairs = int64_t(m->blk[i].T) * m->blk[i].T;
    m->reg_cta_prefix.push_back(m->reg_cta_prefix.back() + (pairs + 127) / 128);
    for (int r = 0; r < m->blk[i].N; ++r) row_blk.push_back(i);
  }
  m->d_blk_mat_off.upload(mo, s);
  m->d_blk_bt_off.upload(bo, s);
  m->d_blk_dof_off.upload(dofo, s);
  m->d_blk_row_off.upload(rowo, s);
  m->d_blk_N.upload(N, s);
  m->d_blk_T.upload(T, s);
  m->d_reg_cta_prefix.upload(m->reg_cta_prefix, s);
  m->d_row_blk.upload(row_blk, s);
  MTF_CUDA(cudaStreamSynchronize(s));
}

}  // namespace mtf
