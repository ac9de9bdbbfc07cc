// Graph set-up: validation of the input CSR (Section 2: simple, undirected,
// positive weights), concatenation of a batch into one block-diagonal CSR,
// generalised degrees, ||L||_1 per graph, row tiles, and the SpMM schedule
// (lanes per row and the list of hub rows).
#include <algorithm>
#include <functional>
#include <climits>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <thread>

#include "internal.h"

namespace lapeig {

namespace {

// Several device arrays carved from one allocation, filled by one copy from a
// host staging buffer (arrays without a source are zero): graph set-up costs
// one cudaMalloc and one cudaMemcpy instead of one pair per array.
struct Packer {
  struct Item { void** dst; const void* src; size_t bytes, off; };
  std::vector<Item> items;
  size_t total = 0;
  template <typename T>
  void add(T** dst, const T* src, size_t count) {
    *dst = nullptr;
    if (count == 0) return;
    total = (total + 255) / 256 * 256;
    items.push_back({reinterpret_cast<void**>(dst), src, count * sizeof(T), total});
    total += count * sizeof(T);
  }
  int upload(void** block) {
    *block = nullptr;
    if (total == 0) return LAP_OK;
    if (cudaMalloc(block, total) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc failed in graph set-up");
      return LAP_ENOMEM;
    }
    std::vector<char> h(total, 0);
    for (const Item& it : items)
      if (it.src) std::memcpy(h.data() + it.off, it.src, it.bytes);
    if (cudaMemcpy(*block, h.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("cudaMemcpy failed in graph set-up");
      return LAP_ECUDA;
    }
    for (const Item& it : items) *it.dst = static_cast<char*>(*block) + it.off;
    return LAP_OK;
  }
};

// Rows [0, n) cut into at most `threads` ranges of about equal nonzero
// count (rowptr quantiles); f(r0, r1, t) runs on each, the calling thread
// taking range 0.  One range (one thread) below ~64k nonzeros.
template <typename F>
void for_row_ranges(int64_t n, const int64_t* rowptr, F&& f) {
  const int64_t nnz = rowptr[n];
  const unsigned hw = std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
  const int nt = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)hw, nnz / 65536));
  std::vector<int64_t> cut((size_t)nt + 1, n);
  cut[0] = 0;
  for (int t = 1; t < nt; ++t)
    cut[(size_t)t] = std::lower_bound(rowptr, rowptr + n + 1, nnz * t / nt) - rowptr;
  for (int t = 1; t <= nt; ++t) cut[(size_t)t] = std::max(cut[(size_t)t], cut[(size_t)t - 1]);
  std::vector<std::thread> th;
  int started = 1;  // ranges 1 .. started-1 have a thread
  try {
    for (int t = 1; t < nt; ++t) {
      th.emplace_back([&, t] { f(cut[(size_t)t], cut[(size_t)t + 1], t); });
      started = t + 1;
    }
  } catch (...) {  // no thread could be created: the caller's thread takes the rest
  }
  for (int t = started; t < nt; ++t) f(cut[(size_t)t], cut[(size_t)t + 1], t);
  f(cut[0], cut[1], 0);
  for (auto& x : th) x.join();
}

int validate(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* w) {
  if (n < 1 || !rowptr || (!colidx && rowptr[n] > 0)) {
    set_error("n < 1 or NULL CSR array");
    return LAP_EINVAL;
  }
  if (rowptr[0] != 0) { set_error("rowptr[0] != 0"); return LAP_EINVAL; }
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) { set_error("rowptr not monotone"); return LAP_EINVAL; }
  const int64_t nnz = rowptr[n];
  if (nnz >= (int64_t(1) << 31) || n >= (int64_t(1) << 31)) { set_error("graph too large for int32 indices"); return LAP_EINVAL; }
  // per-row checks, in parallel; the failure reported is the first in row
  // order (each range keeps its first, the ranges are in row order)
  struct Fail { int64_t row = -1; int code = LAP_OK; const char* msg = nullptr; };
  const unsigned hw = std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
  std::vector<Fail> fails(hw);
  for_row_ranges(n, rowptr, [&](int64_t r0, int64_t r1, int t) {
    for (int64_t i = r0; i < r1; ++i) {
      for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        const int64_t j = colidx[p];
        const char* msg = nullptr;
        int code = LAP_OK;
        if (j < 0 || j >= n) { msg = "column index out of range"; code = LAP_EINVAL; }
        else if (j == i) { msg = "diagonal entry (self-loop) in adjacency"; code = LAP_ESELFLOOP; }
        else if (p > rowptr[i] && colidx[p - 1] >= j) { msg = "column indices not strictly increasing"; code = LAP_EUNSORTED; }
        else if (w && !(std::isfinite(w[p]) && w[p] > 0.0)) { msg = "weight not finite and positive"; code = LAP_EWEIGHT; }
        if (code != LAP_OK) { fails[(size_t)t] = Fail{i, code, msg}; return; }
      }
    }
  });
  for (const Fail& f : fails)
    if (f.code != LAP_OK) { set_error(f.msg); return f.code; }
  // symmetry: (i, j, w) needs (j, i, w).  With sorted rows and no duplicate
  // column, a binary search for i in row j per nonzero decides it: the map
  // (i, j) -> (j, i) then sends the pattern into itself injectively, so onto.
  std::vector<int> bad(hw, 0);  // 1: pattern, 2: values
  // (the lookups are random rows: they go in batches whose row-pointer loads
  // and first column loads are all issued before any search depends on them)
  for_row_ranges(n, rowptr, [&](int64_t r0, int64_t r1, int t) {
    constexpr int kB = 16;
    int64_t rows[kB], js[kB], ps[kB], lo[kB], hi[kB];
    int64_t i = r0;
    const int64_t pend = rowptr[r1];
    for (int64_t p0 = rowptr[r0]; p0 < pend; p0 += kB) {
      const int nb = (int)std::min<int64_t>(kB, pend - p0);
      for (int k = 0; k < nb; ++k) {  // the row of each nonzero
        while (rowptr[i + 1] <= p0 + k) ++i;
        rows[k] = i;
        ps[k] = p0 + k;
        js[k] = colidx[p0 + k];
      }
      for (int k = 0; k < nb; ++k) { lo[k] = rowptr[js[k]]; hi[k] = rowptr[js[k] + 1]; }
      for (int k = 0; k < nb; ++k) __builtin_prefetch(colidx + lo[k]);
      for (int k = 0; k < nb; ++k) {
        const int32_t* b1 = colidx + hi[k];
        const int32_t* q = std::lower_bound(colidx + lo[k], b1, (int32_t)rows[k]);
        if (q == b1 || *q != rows[k]) { bad[(size_t)t] = 1; return; }
        if (w && w[q - colidx] != w[ps[k]]) { bad[(size_t)t] = 2; return; }
      }
    }
  });
  int worst = 0;
  for (int v : bad) worst = worst == 1 ? 1 : (v == 1 ? 1 : std::max(worst, v));
  if (worst == 1) { set_error("adjacency pattern not symmetric"); return LAP_ENOTSYM; }
  if (worst == 2) { set_error("adjacency values not symmetric"); return LAP_ENOTSYM; }
  return LAP_OK;
}

}  // namespace

int graph_set_schedule(lap_graph* g, int team, int long_thresh) {
  if (team != 0) {
    if (team != 4 && team != 8 && team != 16 && team != 32) { set_error("team must be 4, 8, 16 or 32"); return LAP_EINVAL; }
    g->dg.team = team;
  }
  if (long_thresh > 0) g->dg.long_thresh = long_thresh;
  // hub rows: degree above the threshold
  std::vector<int> hubs;
  const int n = g->hg.n;
  for (int i = 0; i < n; ++i)
    if (g->rowptr_h[i + 1] - g->rowptr_h[i] > g->dg.long_thresh) hubs.push_back(i);
  // longest first so the heaviest CTAs start earliest
  std::sort(hubs.begin(), hubs.end(), [&](int a, int b) {
    const int da = g->rowptr_h[a + 1] - g->rowptr_h[a], db = g->rowptr_h[b + 1] - g->rowptr_h[b];
    return da != db ? da > db : a < b;
  });
  cudaFree(g->d_sched);
  g->d_sched = nullptr;
  g->d_long = nullptr; g->d_long_seg = nullptr; g->d_chunks = nullptr; g->d_hub_chunks = nullptr;
  g->d_hub_cnt = nullptr; g->d_hub_part = nullptr; g->d_erp = nullptr; g->d_order = nullptr;
  std::vector<int> erp((size_t)n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const int d = g->rowptr_h[i + 1] - g->rowptr_h[i];
    erp[i + 1] = erp[i] + (d > g->dg.long_thresh ? 0 : d);
  }
  std::vector<int> hseg(hubs.size());
  for (size_t h = 0; h < hubs.size(); ++h)
    hseg[h] = (int)(std::upper_bound(g->row0.begin(), g->row0.end(), hubs[h]) - g->row0.begin()) - 1;
  // chunks of at most kHubChunk nonzeros, hubs in order (longest first)
  std::vector<int4> chunks;
  std::vector<int2> hub_chunks(hubs.size());
  for (size_t h = 0; h < hubs.size(); ++h) {
    const int r = hubs[h], p0 = g->rowptr_h[r], p1 = g->rowptr_h[r + 1];
    hub_chunks[h] = make_int2((int)chunks.size(), (p1 - p0 + kHubChunk - 1) / kHubChunk);
    for (int p = p0; p < p1; p += kHubChunk) chunks.push_back(make_int4(r, p, std::min(p + kHubChunk, p1), (int)h));
  }
  // ordinary rows by decreasing degree, ties by row (a counting sort)
  std::vector<int> order;
  {
    const int lt = g->dg.long_thresh;
    std::vector<int> cnt((size_t)lt + 2, 0);
    for (int i = 0; i < n; ++i) {
      const int d = g->rowptr_h[i + 1] - g->rowptr_h[i];
      if (d <= lt) ++cnt[(size_t)(lt - d) + 1];
    }
    for (size_t v = 1; v < cnt.size(); ++v) cnt[v] += cnt[v - 1];
    order.resize((size_t)cnt.back());
    for (int i = 0; i < n; ++i) {
      const int d = g->rowptr_h[i + 1] - g->rowptr_h[i];
      if (d <= lt) order[(size_t)cnt[(size_t)(lt - d)]++] = i;
    }
  }
  Packer pk;  // hub counters start at zero (no source)
  pk.add(&g->d_order, order.data(), order.size());
  pk.add(&g->d_long, hubs.data(), hubs.size());
  pk.add(&g->d_long_seg, hseg.data(), hseg.size());
  pk.add(&g->d_chunks, chunks.data(), chunks.size());
  pk.add(&g->d_hub_chunks, hub_chunks.data(), hub_chunks.size());
  pk.add<int>(&g->d_hub_cnt, nullptr, hubs.size());
  pk.add<double>(&g->d_hub_part, nullptr, chunks.size() * kPartStride);
  pk.add(&g->d_erp, erp.data(), erp.size());
  const int rc = pk.upload(&g->d_sched);
  if (rc) return rc;
  g->long_rows_h = hubs;
  g->dg.long_rows = g->d_long;
  g->dg.nlong = (int)hubs.size();
  g->dg.chunks = g->d_chunks;
  g->dg.nchunk = (int)chunks.size();
  g->dg.hub_chunks = g->d_hub_chunks;
  g->dg.hub_cnt = g->d_hub_cnt;
  g->dg.hub_part = g->d_hub_part;
  g->dg.erp = g->d_erp;
  g->dg.order = g->d_order;
  g->dg.norder = (int)order.size();
  return LAP_OK;
}

int graph_build(int nb, const int64_t* n, const int64_t* const* rowptr, const int32_t* const* colidx,
                const double* const* weights, lap_graph** out, bool check) {
  *out = nullptr;
  if (nb < 1 || !n || !rowptr || !colidx) { set_error("bad batch arguments"); return LAP_EINVAL; }
  int64_t ntot = 0, nnztot = 0;
  bool weighted = false;
  for (int s = 0; s < nb; ++s) {
    if (!rowptr[s]) { set_error("NULL rowptr"); return LAP_EINVAL; }
    if (check) {  // (a handle's own relabelled copy is valid by construction)
      const int rc = validate(n[s], rowptr[s], colidx[s], weights ? weights[s] : nullptr);
      if (rc) return rc;
    }
    ntot += n[s];
    nnztot += rowptr[s][n[s]];
    if (weights && weights[s]) weighted = true;
  }
  if (ntot >= (int64_t(1) << 31) || nnztot >= (int64_t(1) << 31)) { set_error("batch too large for int32 indices"); return LAP_EINVAL; }

  lap_graph* g = new lap_graph();
  g->hg.n = (int)ntot;
  g->hg.nseg = nb;
  g->hg.nnz = nnztot;
  g->hg.weighted = weighted ? 1 : 0;

  std::vector<int> colcat((size_t)nnztot);
  std::vector<double> w64(weighted ? (size_t)nnztot : 0);
  std::vector<double> deg((size_t)ntot);
  g->rowptr_h.assign((size_t)ntot + 1, 0);
  g->row0.assign(nb + 1, 0);
  g->norm1.assign(nb, 0.0);
  int64_t r = 0, p = 0;
  int maxdeg = 0;
  const unsigned hw = std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
  for (int s = 0; s < nb; ++s) {
    g->row0[s] = (int)r;
    const int64_t* rp = rowptr[s];
    const double* ws = weights ? weights[s] : nullptr;
    const int64_t rb = r, pb = p;  // the graph's first row and nonzero in the concatenation
    std::vector<double> dmax_t(hw, 0.0);
    std::vector<int> maxdeg_t(hw, 0);
    for_row_ranges(n[s], rp, [&](int64_t i0, int64_t i1, int t) {
      double dm = 0.0;
      int md = 0;
      for (int64_t i = i0; i < i1; ++i) {
        double d = 0.0;
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
          colcat[(size_t)(pb + q)] = (int)(colidx[s][q] + rb);
          const double wv = ws ? ws[q] : 1.0;
          if (weighted) w64[(size_t)(pb + q)] = wv;
          d += wv;
        }
        g->rowptr_h[(size_t)(rb + i + 1)] = (int)(pb + rp[i + 1]);
        deg[(size_t)(rb + i)] = d;
        dm = std::max(dm, d);
        md = std::max(md, (int)(rp[i + 1] - rp[i]));
      }
      dmax_t[(size_t)t] = dm;
      maxdeg_t[(size_t)t] = md;
    });
    r += n[s];
    p += rp[n[s]];
    double dmax = 0.0;
    for (unsigned t = 0; t < hw; ++t) {
      dmax = std::max(dmax, dmax_t[t]);
      maxdeg = std::max(maxdeg, maxdeg_t[t]);
    }
    g->norm1[s] = 2.0 * dmax;
  }
  g->row0[nb] = (int)r;
  g->avg_degree = ntot ? (double)nnztot / (double)ntot : 0.0;
  g->max_degree = maxdeg;

  // tiles: every phase of the persistent correction solve ends at a grid
  // barrier, so the CTAs must get equal work.  A row costs its SpMM work (its
  // length; a hub row, longer than the default threshold 64, nothing: its
  // nonzeros go to chunks) plus 8 for the row-wise phases.  A single graph of
  // more than 4,096 rows is cut into a multiple of 304 (= 2 CTAs x 152 SMs)
  // tiles of equal cost (at most 256 rows each).
  std::vector<Tile> tiles;
  g->tile_ptr.assign(nb + 1, 0);
  for (int s = 0; s < nb; ++s) {
    g->tile_ptr[s] = (int)tiles.size();
    const int a0 = g->row0[s], a1 = g->row0[s + 1], ns = a1 - a0;
    auto cost = [&](int r) {
      const int d = g->rowptr_h[r + 1] - g->rowptr_h[r];
      return (int64_t)(d > 64 ? 0 : d) + 8;
    };
    int64_t total = 0;
    for (int r = a0; r < a1; ++r) total += cost(r);
    if (nb == 1 && ns > 4096) {
      // T tiles (a multiple of 304, with headroom so the row cap rarely
      // binds), cut at the cost quantiles k * total / T
      const int64_t want = (ns + kTileRows - 1) / kTileRows;
      const int64_t T = std::max<int64_t>(1, (want * 5 / 4 + 303) / 304) * 304;
      // With no more hub chunks (of at most kHubChunk nonzeros, hubs longest
      // first) than tiles, the correction solve hands chunk i to CTA i, which
      // holds tile i: the chunk's gathers plus its completion (about 100 row
      // units, measured) count against tile i's budget.
      std::vector<int> hub_deg;
      for (int r = a0; r < a1; ++r)
        if (g->rowptr_h[r + 1] - g->rowptr_h[r] > 64) hub_deg.push_back(g->rowptr_h[r + 1] - g->rowptr_h[r]);
      std::sort(hub_deg.begin(), hub_deg.end(), std::greater<int>());
      std::vector<int64_t> xpre((size_t)T + 1, 0);  // prefix sums of the chunk costs per tile
      int64_t nchunk = 0;
      for (int d : hub_deg) nchunk += (d + kHubChunk - 1) / kHubChunk;
      if (nchunk <= T) {
        int64_t i = 0;
        for (int d : hub_deg)
          for (int q0 = 0; q0 < d; q0 += kHubChunk, ++i) xpre[(size_t)i + 1] = std::min(kHubChunk, d - q0) + 100;
        for (int64_t k = 1; k <= T; ++k) xpre[(size_t)k] += xpre[(size_t)k - 1];
      }
      const int64_t work = total + xpre[(size_t)T];
      int idx = 0, a = a0;
      int64_t cum = 0;
      for (int64_t kq = 1; kq <= T && a < a1; ++kq) {
        const int64_t goal = (kq == T) ? INT64_MAX : (work * kq + T - 1) / T - xpre[(size_t)kq];
        int e = a;
        while (e < a1 && e - a < kTileRows && (e == a || cum < goal)) cum += cost(e++);
        tiles.push_back(Tile{s, a, e, idx++});
        a = e;
      }
      while (a < a1) {  // only if the row cap bound somewhere
        const int e = std::min(a + kTileRows, a1);
        tiles.push_back(Tile{s, a, e, idx++});
        a = e;
      }
    } else {
      // a batch (many tiles per CTA) or a small graph: rows per tile from the
      // graph size (several CTAs per SM), cut early at twice the mean cost
      int rows = (ns + 4 * 152 - 1) / (4 * 152);
      rows = std::max(64, std::min((rows + 31) / 32 * 32, kTileRows));
      const int64_t budget = std::max<int64_t>(64, 2 * total * rows / std::max(ns, 1));
      int idx = 0, a = a0;
      while (a < a1) {
        int e = a;
        int64_t w = 0;
        while (e < a1 && e - a < rows && (e == a || w < budget)) w += cost(e++);
        tiles.push_back(Tile{s, a, e, idx++});
        a = e;
      }
    }
  }
  g->tile_ptr[nb] = (int)tiles.size();
  g->hg.ntiles = (int)tiles.size();

  std::vector<float> w32(w64.begin(), w64.end());
  std::vector<float> deg32(deg.begin(), deg.end());
  g->colidx_h = std::move(colcat);  // kept for set-ups that need the pattern (preconditioner)
  g->w64_h = w64;
  Packer pk;
  pk.add(&g->d_rowptr, g->rowptr_h.data(), g->rowptr_h.size());
  pk.add(&g->d_colidx, g->colidx_h.data(), g->colidx_h.size());
  if (weighted) {
    pk.add(&g->d_w64, w64.data(), w64.size());
    pk.add(&g->d_w32, w32.data(), w32.size());
  }
  pk.add(&g->d_deg64, deg.data(), deg.size());
  pk.add(&g->d_deg32, deg32.data(), deg32.size());
  pk.add(&g->d_row0, g->row0.data(), g->row0.size());
  pk.add(&g->d_norm1, g->norm1.data(), g->norm1.size());
  pk.add(&g->d_tiles, tiles.data(), tiles.size());
  pk.add(&g->d_tile_ptr, g->tile_ptr.data(), g->tile_ptr.size());
  // reduction scratch, zero at rest (no source: zero-filled)
  g->red.stride = 4608;
  pk.add<double>(&g->red.acc, nullptr, (size_t)nb * g->red.stride);
  pk.add<int>(&g->red.counter, nullptr, (size_t)nb);
  int rc = pk.upload(&g->d_block);
  if (rc) { graph_free(g); return rc; }

  DevGraph& d = g->dg;
  d.n = (int)ntot;
  d.nseg = nb;
  d.nnz = nnztot;
  d.rowptr = g->d_rowptr;
  d.colidx = g->d_colidx;
  d.w32 = g->d_w32;
  d.w64 = g->d_w64;
  d.deg64 = g->d_deg64;
  d.deg32 = g->d_deg32;
  d.row0 = g->d_row0;
  d.tiles = g->d_tiles;
  d.ntiles = (int)tiles.size();
  d.tile_ptr = g->d_tile_ptr;
  d.counters = g->red.counter;
  // schedule heuristic (overridden by the autotuner or the caller)
  d.team = g->avg_degree <= 6.0 ? 4 : (g->avg_degree <= 24.0 ? 8 : (g->avg_degree <= 96.0 ? 16 : 32));
  d.long_thresh = 64;
  d.vec_u = 4;
  rc = graph_set_schedule(g, 0, 0);
  if (rc) { graph_free(g); return rc; }
  *out = g;
  return LAP_OK;
}

void graph_free(lap_graph* g) {
  if (!g) return;
  cudaFree(g->d_block);  // every array of the graph
  cudaFree(g->d_sched);  // the hub schedule
  cudaFree(g->d_prec);   // the preconditioner
  cudaFree(g->scratch); cudaFree(g->small);
  cudaFree(g->d_perm_of_parent);
  g->pcg.release();
  graph_free(g->twin);
  delete g;
}

unsigned long long timeout_ns_of(double opts_ms, double handle_ms) {
  const double ms = opts_ms > 0.0 ? opts_ms : (handle_ms > 0.0 ? handle_ms : 0.0);
  if (ms <= 0.0) return kDefaultTimeoutNs;
  const double ns = ms * 1e6;
  return ns >= 1.8e19 ? ~0ull : (ns < 1.0 ? 1ull : (unsigned long long)ns);
}

int graph_scratch(lap_graph* g, size_t bytes, size_t small_bytes) {
  if (bytes > g->scratch_bytes) {
    cudaFree(g->scratch);
    g->scratch = nullptr;
    g->scratch_bytes = 0;
    if (cudaMalloc(&g->scratch, bytes) != cudaSuccess) { cudaGetLastError(); set_error("scratch allocation failed"); return LAP_ENOMEM; }
    g->scratch_bytes = bytes;
  }
  if (small_bytes > g->small_bytes) {
    cudaFree(g->small);
    g->small = nullptr;
    g->small_bytes = 0;
    if (cudaMalloc(reinterpret_cast<void**>(&g->small), small_bytes) != cudaSuccess) { cudaGetLastError(); set_error("scratch allocation failed"); return LAP_ENOMEM; }
    g->small_bytes = small_bytes;
  }
  return LAP_OK;
}

}  // namespace lapeig

namespace lapeig {

int PcgWork::init(int nseg_) {
  nseg = nseg_;
  const size_t a = (size_t)nseg * acc_stride;
  const size_t st = (size_t)nseg * 64;
  bytes = sizeof(double) * (4 * a + 2 * st + 2 * st) + sizeof(int) * 2 * st + 64;
  char* base = nullptr;
  if (cudaMalloc(reinterpret_cast<void**>(&base), bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("PCG workspace allocation failed");
    return LAP_ENOMEM;
  }
  if (cudaMemset(base, 0, bytes) != cudaSuccess) { set_error("cudaMemset failed"); cudaFree(base); return LAP_ECUDA; }
  acc1 = reinterpret_cast<double*>(base);
  acc2 = acc1 + 2 * a;
  rho = acc2 + 2 * a;
  res0 = rho + 2 * st;
  resn = res0 + st;
  done = reinterpret_cast<int*>(resn + st);
  bar = reinterpret_cast<unsigned*>(done + 2 * st);
  return LAP_OK;
}

void PcgWork::release() {
  cudaFree(acc1);
  acc1 = nullptr;
}

FusedPcg PcgWork::args(const void* X, int ldx, const void* R, int ldr, void* Tt, void* RES, void* Z, void* P, void* AP,
                       void* LX, int ldlx, int ld, int b, const double* theta, int64_t sth, const int* active, const int* seg_skip,
                       double delta, int itmax, const int* hub_seg) const {
  FusedPcg f;
  f.Xv = X; f.ldx = ldx; f.Rv = R; f.ldr = ldr; f.Ttv = Tt; f.RESv = RES; f.Zv = Z; f.Pv = P; f.APv = AP;
  f.LXv = LX; f.ldlx = ldlx;
  f.ld = ld; f.b = b; f.theta = theta; f.sth = sth; f.active = active; f.bstride = 64; f.seg_skip = seg_skip;
  f.delta = delta; f.itmax = itmax; f.acc1 = acc1; f.acc2 = acc2; f.acc_stride = acc_stride; f.rho = rho;
  f.done = done; f.res0 = res0; f.resn = resn; f.state_stride = (int64_t)nseg * 64; f.hub_seg = hub_seg;
  f.bar = gridbar();
  f.iters_out = reinterpret_cast<int*>(bar + 3);
  f.stop = reinterpret_cast<int*>(bar + 4);
  f.split_rows = split_rows;
  return f;
}

int PcgWork::steps_done(cudaStream_t s) const {
  int v = 0;
  cudaMemcpyAsync(&v, bar + 3, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return v;
}

void PcgWork::status(cudaStream_t s, int* err, int* steps) const {
  int v[2] = {0, 0};
  cudaMemcpyAsync(v, bar + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (v[0]) reset(s);
  if (err) *err = v[0];
  if (steps) *steps = v[1];
}

int PcgWork::error_flag(cudaStream_t s) const {
  int e = 0;
  cudaMemcpyAsync(&e, bar + 2, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (e) reset(s);
  return e;
}

void PcgWork::reset(cudaStream_t s) const {
  if (acc1) cudaMemsetAsync(acc1, 0, bytes, s);
  // a CTA that passed a barrier before the flag was set may have left a hub
  // row with only some of its chunks counted
  if (hub_cnt && nlong > 0) cudaMemsetAsync(hub_cnt, 0, sizeof(int) * (size_t)nlong, s);
  cudaStreamSynchronize(s);
}

}  // namespace lapeig
