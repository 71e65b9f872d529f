// sx_remesh.cpp -- host side of the dynamic grid update (Sect. 2.1.4):
// removes an independent set of vertices from a Delaunay tetrahedralisation
// by re-triangulating their cavities, and patches the graph (CSR), the cell
// volumes and the tetrahedra.
//
// Removing vertex v leaves a cavity, the union of the tetrahedra around v.
// The tetrahedra outside keep their empty circumspheres, so the cavity is
// filled by the Delaunay tetrahedra of v's neighbours (its link) that lie in
// it.  The link's Delaunay tetrahedralisation is built here by Bowyer-Watson
// insertion (tens of points), in coordinates relative to v; its tetrahedra
// whose centroid lies in one of v's tetrahedra are kept, and they must fill
// the cavity's volume (else the call reports the cavity and the caller
// rebuilds the grid).  No two removed vertices are adjacent, so no
// tetrahedron holds two of them and the cavities are filled independently.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <new>
#include <stdexcept>
#include <system_error>
#include <thread>
#include <vector>

#include "simplexgb.h"

namespace {

struct V3 {
  double x, y, z;
};
inline V3 sub(const V3 &a, const V3 &b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline double dot(const V3 &a, const V3 &b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(const V3 &a, const V3 &b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
// 6 x the signed volume of (a, b, c, d): positive when d is on the side of
// (a, b, c) that the right-hand rule points to
inline double orient(const V3 &a, const V3 &b, const V3 &c, const V3 &d) {
  return dot(cross(sub(b, a), sub(c, a)), sub(d, a));
}
// > 0 when e lies inside the circumsphere of the positively oriented (a, b, c, d)
double insphere(const V3 &a, const V3 &b, const V3 &c, const V3 &d, const V3 &e) {
  const V3 pa = sub(a, e), pb = sub(b, e), pc = sub(c, e), pd = sub(d, e);
  const double la = dot(pa, pa), lb = dot(pb, pb), lc = dot(pc, pc), ld = dot(pd, pd);
  // D = det of the 4 x 4 matrix with rows (p, |p|^2), by cofactors along the
  // last column: D = -la det(pb,pc,pd) + lb det(pa,pc,pd) - lc det(pa,pb,pd)
  // + ld det(pa,pb,pc); for a positively oriented tetrahedron D < 0 exactly
  // when e is inside, so the result is -D
  const double ob = dot(cross(pc, pd), pb), oa = dot(cross(pc, pd), pa), oc = dot(cross(pb, pd), pa),
               od = dot(cross(pb, pc), pa);
  return la * ob - lb * oa + lc * oc - ld * od;
}

struct Tet {
  int v[4];
};

// Delaunay tetrahedralisation of m points by Bowyer-Watson insertion into a
// bounding tetrahedron; tetrahedra are kept positively oriented.  Returns the
// tetrahedra of the points (those without a bounding vertex).
bool delaunay_small(const std::vector<V3> &pts, std::vector<Tet> &out) {
  const int m = (int)pts.size();
  double r = 0.0;
  for (const V3 &p : pts) r = std::max(r, std::sqrt(dot(p, p)));
  if (!(r > 0.0)) return false;
  std::vector<V3> P(pts);
  const double s = 64.0 * r;  // the bounding tetrahedron, far outside
  P.push_back({-s, -s, -s});
  P.push_back({3 * s, -s, -s});
  P.push_back({-s, 3 * s, -s});
  P.push_back({-s, -s, 3 * s});
  std::vector<Tet> T;
  T.push_back({{m, m + 1, m + 2, m + 3}});
  if (orient(P[m], P[m + 1], P[m + 2], P[m + 3]) < 0) std::swap(T[0].v[0], T[0].v[1]);
  std::vector<char> bad;
  struct Face {
    int a, b, c;  // as oriented in its tetrahedron
    int key[3];   // the same vertices, ascending
  };
  std::vector<Face> faces;
  for (int i = 0; i < m; ++i) {
    bad.assign(T.size(), 0);
    bool any = false;
    for (size_t t = 0; t < T.size(); ++t) {
      const Tet &q = T[t];
      if (insphere(P[q.v[0]], P[q.v[1]], P[q.v[2]], P[q.v[3]], P[i]) > 0) {
        bad[t] = 1;
        any = true;
      }
    }
    if (!any) return false;
    // the cavity's boundary: faces of bad tetrahedra not shared with another
    // bad one (a shared face appears twice among them), oriented outward
    faces.clear();
    for (size_t t = 0; t < T.size(); ++t) {
      if (!bad[t]) continue;
      const int *v = T[t].v;
      const int f[4][3] = {{v[1], v[2], v[3]}, {v[0], v[3], v[2]}, {v[0], v[1], v[3]}, {v[0], v[2], v[1]}};
      for (int k = 0; k < 4; ++k) {
        Face fc{f[k][0], f[k][1], f[k][2], {f[k][0], f[k][1], f[k][2]}};
        std::sort(fc.key, fc.key + 3);
        faces.push_back(fc);
      }
    }
    std::sort(faces.begin(), faces.end(), [](const Face &x, const Face &y) {
      return std::lexicographical_compare(x.key, x.key + 3, y.key, y.key + 3);
    });
    {
      size_t w = 0;
      for (size_t k = 0; k < faces.size();) {
        size_t e = k + 1;
        while (e < faces.size() && std::equal(faces[e].key, faces[e].key + 3, faces[k].key)) ++e;
        if (e - k == 1) faces[w++] = faces[k];
        k = e;
      }
      faces.resize(w);
    }
    std::vector<Tet> keep;
    keep.reserve(T.size() + faces.size());
    for (size_t t = 0; t < T.size(); ++t)
      if (!bad[t]) keep.push_back(T[t]);
    for (const Face &f : faces) {
      // (a, b, c) faces outward from the removed tetrahedron's interior, so
      // the new point on its inner side gives orient(a, c, b, i) > 0
      Tet q{{f.a, f.c, f.b, i}};
      if (!(orient(P[q.v[0]], P[q.v[1]], P[q.v[2]], P[q.v[3]]) > 0)) return false;
      keep.push_back(q);
    }
    T.swap(keep);
  }
  out.clear();
  for (const Tet &q : T)
    if (q.v[0] < m && q.v[1] < m && q.v[2] < m && q.v[3] < m) out.push_back(q);
  return true;
}

// Whether point p lies in tetrahedron (a, b, c, d) (barycentric, with slack).
bool in_tet(const V3 &p, const V3 &a, const V3 &b, const V3 &c, const V3 &d) {
  const double vol = orient(a, b, c, d);
  if (vol == 0.0) return false;
  const double eps = -1e-9 * std::fabs(vol);
  const double l0 = orient(p, b, c, d), l1 = orient(a, p, c, d), l2 = orient(a, b, p, d),
               l3 = orient(a, b, c, p);
  if (vol > 0) return l0 >= eps && l1 >= eps && l2 >= eps && l3 >= eps;
  return l0 <= -eps && l1 <= -eps && l2 <= -eps && l3 <= -eps;
}

double tet_volume(const double *pos, const int32_t *t) {
  const V3 a{pos[3 * (int64_t)t[0]], pos[3 * (int64_t)t[0] + 1], pos[3 * (int64_t)t[0] + 2]};
  const V3 b{pos[3 * (int64_t)t[1]], pos[3 * (int64_t)t[1] + 1], pos[3 * (int64_t)t[1] + 2]};
  const V3 c{pos[3 * (int64_t)t[2]], pos[3 * (int64_t)t[2] + 1], pos[3 * (int64_t)t[2] + 2]};
  const V3 d{pos[3 * (int64_t)t[3]], pos[3 * (int64_t)t[3] + 1], pos[3 * (int64_t)t[3] + 2]};
  return std::fabs(orient(a, b, c, d)) / 6.0;
}

// Runs fn(0) .. fn(nth - 1) on threads; a range whose thread the system
// refuses runs on the calling thread.  fn must not throw.
template <class F>
void run_threads(unsigned nth, F &&fn) {
  std::vector<std::thread> pool;
  pool.reserve(nth);
  unsigned started = 0;
  try {
    for (; nth > 1 && started < nth; ++started) pool.emplace_back(std::ref(fn), started);
  } catch (const std::system_error &) {
  }
  for (unsigned th = started; th < nth; ++th) fn(th);
  for (std::thread &t : pool) t.join();
}

unsigned hardware_threads() { return std::max(1u, std::min(16u, std::thread::hardware_concurrency())); }

// Threads for a pass over `count` items: one per 2^16 items, at most 16.
unsigned pass_threads(int64_t count) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(hardware_threads(), count >> 16));
}

// Start of range th of nth contiguous ranges over [0, count).
inline int64_t range_start(int64_t count, unsigned th, unsigned nth) {
  return count * (int64_t)th / (int64_t)nth;
}

}  // namespace

extern "C" int sx_remesh_remove(int64_t n, const double *pos, const int64_t *row_ptr, const int32_t *col,
                                int64_t ntet, const int32_t *tets, const double *volume, int64_t nrem,
                                const int32_t *removed, sx_remesh_result *out) {
  if (!out) return SX_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->bad_vertex = -1;
  if (n < 1 || !pos || !row_ptr || !col || !volume || (ntet > 0 && !tets) || nrem < 0 ||
      (nrem > 0 && !removed))
    return SX_EINVAL;
  try {
    // the graph and the tetrahedra index the arrays below: check them first
    if (row_ptr[0] != 0) return SX_EINVAL;
    for (int64_t v = 0; v < n; ++v)
      if (row_ptr[v + 1] < row_ptr[v]) return SX_EINVAL;
    const int64_t nnz = row_ptr[n];
    {
      const unsigned nt = pass_threads(nnz + 4 * ntet);
      std::vector<char> bad(nt, 0);
      run_threads(nt, [&](unsigned th) {
        for (int64_t e = range_start(nnz, th, nt), e1 = range_start(nnz, th + 1, nt); e < e1; ++e)
          if (col[e] < 0 || col[e] >= n) {
            bad[th] = 1;
            return;
          }
        for (int64_t i = range_start(4 * ntet, th, nt), i1 = range_start(4 * ntet, th + 1, nt); i < i1; ++i)
          if (tets[i] < 0 || tets[i] >= n) {
            bad[th] = 1;
            return;
          }
      });
      for (char b : bad)
        if (b) return SX_EINVAL;
    }
    std::vector<char> rem((size_t)n, 0);
    for (int64_t k = 0; k < nrem; ++k) {
      if (removed[k] < 0 || removed[k] >= n) return SX_EINVAL;
      rem[(size_t)removed[k]] = 1;
    }
    // the star of every removed vertex
    std::vector<int64_t> cav_of((size_t)n, -1);
    std::vector<int32_t> vs;
    for (int64_t v = 0; v < n; ++v)
      if (rem[(size_t)v]) {
        cav_of[(size_t)v] = (int64_t)vs.size();
        vs.push_back((int32_t)v);
      }
    const size_t ncav = vs.size();
    // the tetrahedra with a removed corner, found by threads over ranges of
    // tetrahedra; each star lists its tetrahedra in ascending order
    std::vector<int64_t> star_cnt(ncav + 1, 0);
    std::vector<char> tet_hit((size_t)ntet, 0);
    std::vector<int64_t> star;
    {
      const unsigned nt = pass_threads(ntet);
      std::vector<std::vector<int64_t>> hits(nt);
      std::vector<char> adjacent(nt, 0), oom(nt, 0);
      run_threads(nt, [&](unsigned th) {
        try {
          for (int64_t t = range_start(ntet, th, nt), t1 = range_start(ntet, th + 1, nt); t < t1; ++t) {
            int h = 0;
            for (int k = 0; k < 4; ++k) h += rem[(size_t)tets[4 * t + k]];
            if (h > 1) {  // removed vertices must not be adjacent
              adjacent[th] = 1;
              return;
            }
            if (h == 1) {
              tet_hit[(size_t)t] = 1;
              hits[th].push_back(t);
            }
          }
        } catch (const std::exception &) {
          oom[th] = 1;
        }
      });
      for (unsigned th = 0; th < nt; ++th) {
        if (oom[th]) return SX_ENOMEM;
        if (adjacent[th]) return SX_EINVAL;
      }
      auto cavity = [&](int64_t t) {
        for (int k = 0; k < 4; ++k)
          if (rem[(size_t)tets[4 * t + k]]) return cav_of[(size_t)tets[4 * t + k]];
        return (int64_t)-1;
      };
      for (const auto &hv : hits)
        for (int64_t t : hv) ++star_cnt[(size_t)cavity(t) + 1];
      for (size_t c = 0; c < ncav; ++c) star_cnt[c + 1] += star_cnt[c];
      star.resize((size_t)star_cnt[ncav]);
      std::vector<int64_t> fill(star_cnt.begin(), star_cnt.end() - 1);
      for (const auto &hv : hits)
        for (int64_t t : hv) star[(size_t)fill[(size_t)cavity(t)]++] = t;
    }
    // fill every cavity: threads take contiguous ranges of cavities, and their
    // tetrahedra are joined in cavity order (the result does not depend on
    // the thread count)
    const unsigned nth = ncav < 64 ? 1u : std::min<unsigned>(hardware_threads(), (unsigned)(ncav / 32));
    std::vector<std::vector<int32_t>> part(nth);
    std::vector<int32_t> failed(nth, -1);
    std::vector<char> no_memory(nth, 0);
    auto fill_range = [&](unsigned th) {
      try {
        const size_t c0 = ncav * th / nth, c1 = ncav * (th + 1) / nth;
        std::vector<int32_t> &nt = part[th];
        std::vector<V3> lp;
        std::vector<int32_t> link;
        std::vector<Tet> dt;
        for (size_t c = c0; c < c1; ++c) {
          const int32_t v = vs[c];
          const V3 o{pos[3 * (int64_t)v], pos[3 * (int64_t)v + 1], pos[3 * (int64_t)v + 2]};
          link.clear();
          double vol_old = 0.0;
          for (int64_t s = star_cnt[c]; s < star_cnt[c + 1]; ++s) {
            const int32_t *q = tets + 4 * star[(size_t)s];
            vol_old += tet_volume(pos, q);
            for (int k = 0; k < 4; ++k)
              if (q[k] != v) link.push_back(q[k]);
          }
          std::sort(link.begin(), link.end());
          link.erase(std::unique(link.begin(), link.end()), link.end());
          lp.resize(link.size());
          for (size_t i = 0; i < link.size(); ++i)
            lp[i] = {pos[3 * (int64_t)link[i]] - o.x, pos[3 * (int64_t)link[i] + 1] - o.y,
                     pos[3 * (int64_t)link[i] + 2] - o.z};
          bool ok = link.size() >= 4 && delaunay_small(lp, dt);
          double vol_new = 0.0;
          for (size_t k = 0; ok && k < dt.size(); ++k) {
            const Tet &q = dt[k];
            const V3 cen{(lp[q.v[0]].x + lp[q.v[1]].x + lp[q.v[2]].x + lp[q.v[3]].x) / 4,
                         (lp[q.v[0]].y + lp[q.v[1]].y + lp[q.v[2]].y + lp[q.v[3]].y) / 4,
                         (lp[q.v[0]].z + lp[q.v[1]].z + lp[q.v[2]].z + lp[q.v[3]].z) / 4};
            bool inside = false;
            for (int64_t s = star_cnt[c]; s < star_cnt[c + 1] && !inside; ++s) {
              const int32_t *w = tets + 4 * star[(size_t)s];
              V3 p4[4];
              for (int a = 0; a < 4; ++a)
                p4[a] = {pos[3 * (int64_t)w[a]] - o.x, pos[3 * (int64_t)w[a] + 1] - o.y,
                         pos[3 * (int64_t)w[a] + 2] - o.z};
              inside = in_tet(cen, p4[0], p4[1], p4[2], p4[3]);
            }
            if (!inside) continue;
            const int32_t g[4] = {link[q.v[0]], link[q.v[1]], link[q.v[2]], link[q.v[3]]};
            vol_new += tet_volume(pos, g);
            nt.insert(nt.end(), g, g + 4);
          }
          if (!ok || !(std::fabs(vol_new - vol_old) <= 1e-9 * vol_old)) {
            failed[th] = v;
            return;
          }
        }
      } catch (const std::exception &) {  // an exception must not leave a thread
        no_memory[th] = 1;
      }
    };
    run_threads(nth, fill_range);
    for (unsigned th = 0; th < nth; ++th)
      if (no_memory[th]) return SX_ENOMEM;
    for (unsigned th = 0; th < nth; ++th)
      if (failed[th] >= 0) {
        out->bad_vertex = failed[th];
        return SX_EINVAL;
      }
    std::vector<int32_t> new_tets;
    {
      size_t tot = 0;
      for (const auto &pv : part) tot += pv.size();
      new_tets.reserve(tot);
      for (const auto &pv : part) new_tets.insert(new_tets.end(), pv.begin(), pv.end());
    }
    const int64_t nnew = (int64_t)new_tets.size() / 4;
    // new edges per vertex (both directions), sorted and unique: one list per
    // link vertex (add_idx: its list, or -1), laid out by counting
    std::vector<int32_t> add_idx((size_t)n, -1);
    std::vector<int64_t> add_ptr(1, 0);
    for (int64_t i = 0; i < 4 * nnew; ++i) {
      const int32_t u = new_tets[(size_t)i];
      if (add_idx[(size_t)u] < 0) {
        add_idx[(size_t)u] = (int32_t)(add_ptr.size() - 1);
        add_ptr.push_back(0);
      }
      add_ptr[(size_t)add_idx[(size_t)u] + 1] += 3;
    }
    const size_t nlink = add_ptr.size() - 1;
    for (size_t k = 0; k < nlink; ++k) add_ptr[k + 1] += add_ptr[k];
    std::vector<int32_t> add_col((size_t)add_ptr[nlink]);
    {
      std::vector<int64_t> fill(add_ptr.begin(), add_ptr.end() - 1);
      for (int64_t t = 0; t < nnew; ++t)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b)
            if (a != b) add_col[(size_t)fill[(size_t)add_idx[(size_t)new_tets[4 * t + a]]]++] = new_tets[4 * t + b];
    }
    std::vector<int64_t> add_len(nlink);  // each list sorted, its unique entries first
    {
      const unsigned nt = pass_threads(add_ptr[nlink]);
      run_threads(nt, [&](unsigned th) {
        for (int64_t k = range_start((int64_t)nlink, th, nt), k1 = range_start((int64_t)nlink, th + 1, nt); k < k1; ++k) {
          int32_t *b = add_col.data() + add_ptr[(size_t)k], *e = add_col.data() + add_ptr[(size_t)k + 1];
          std::sort(b, e);
          add_len[(size_t)k] = std::unique(b, e) - b;
        }
      });
    }
    // renumbering of the survivors, in their old order
    std::vector<int32_t> new_of_old((size_t)n, -1);
    int64_t n2 = 0;
    for (int64_t v = 0; v < n; ++v)
      if (!rem[(size_t)v]) new_of_old[(size_t)v] = (int32_t)n2++;
    // the outputs, allocated once at their final size (the graph at an upper
    // bound, trimmed at the end)
    size_t nadd = 0;
    for (int64_t len : add_len) nadd += (size_t)len;
    const int64_t ntet2 = ntet - (int64_t)star.size() + nnew;
    out->row_ptr = static_cast<int64_t *>(std::malloc(sizeof(int64_t) * ((size_t)n2 + 1)));
    out->col = static_cast<int32_t *>(std::malloc(sizeof(int32_t) * ((size_t)nnz + nadd + 1)));
    out->volume = static_cast<double *>(std::malloc(sizeof(double) * ((size_t)n2 + 1)));
    out->old_of_new = static_cast<int32_t *>(std::malloc(sizeof(int32_t) * ((size_t)n2 + 1)));
    out->tets = static_cast<int32_t *>(std::malloc(sizeof(int32_t) * (4 * (size_t)ntet2 + 1)));
    if (!out->row_ptr || !out->col || !out->volume || !out->old_of_new || !out->tets) {
      sx_remesh_free(out);
      return SX_ENOMEM;
    }
    // the graph: each survivor's row without removed neighbours, merged with
    // its new neighbours (both ascending); threads over ranges of vertices
    // count the rows, then write them at their offsets
    int64_t *rp2 = out->row_ptr;
    int32_t *col2 = out->col;
    auto merge_row = [&](int64_t v, auto &&emit) {
      const int32_t *a = nullptr, *a1 = nullptr;  // v's new neighbours, ascending
      if (add_idx[(size_t)v] >= 0) {
        a = add_col.data() + add_ptr[(size_t)add_idx[(size_t)v]];
        a1 = a + add_len[(size_t)add_idx[(size_t)v]];
      }
      for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        const int32_t w = col[e];
        for (; a < a1 && *a < w; ++a)
          if (!rem[(size_t)*a]) emit(new_of_old[(size_t)*a]);
        if (a < a1 && *a == w) ++a;  // already an edge
        if (!rem[(size_t)w]) emit(new_of_old[(size_t)w]);
      }
      for (; a < a1; ++a)
        if (!rem[(size_t)*a]) emit(new_of_old[(size_t)*a]);
    };
    const unsigned ntg = pass_threads(nnz);
    rp2[0] = 0;
    run_threads(ntg, [&](unsigned th) {
      for (int64_t v = range_start(n, th, ntg), v1 = range_start(n, th + 1, ntg); v < v1; ++v) {
        if (rem[(size_t)v]) continue;
        int64_t len = 0;
        merge_row(v, [&](int32_t) { ++len; });
        rp2[(size_t)new_of_old[(size_t)v] + 1] = len;
      }
    });
    for (int64_t i = 0; i < n2; ++i) rp2[i + 1] += rp2[i];
    run_threads(ntg, [&](unsigned th) {
      for (int64_t v = range_start(n, th, ntg), v1 = range_start(n, th + 1, ntg); v < v1; ++v) {
        if (rem[(size_t)v]) continue;
        int64_t m = rp2[(size_t)new_of_old[(size_t)v]];
        merge_row(v, [&](int32_t w) { col2[m++] = w; });
      }
    });
    const int64_t m = rp2[n2];
    if (int32_t *shrunk = static_cast<int32_t *>(std::realloc(out->col, sizeof(int32_t) * ((size_t)m + 1))))
      out->col = shrunk;
    // cell volumes: each survivor's old volume, then a quarter of each old
    // cavity tetrahedron leaves its surviving corners and a quarter of each
    // new one joins its corners (all survivors: the link of a removed vertex
    // holds no removed vertex)
    run_threads(pass_threads(n), [&, nt = pass_threads(n)](unsigned th) {
      for (int64_t v = range_start(n, th, nt), v1 = range_start(n, th + 1, nt); v < v1; ++v) {
        const int32_t w = new_of_old[(size_t)v];
        if (w < 0) continue;
        out->volume[w] = volume[v];
        out->old_of_new[w] = (int32_t)v;
      }
    });
    for (size_t s = 0; s < star.size(); ++s) {
      const int32_t *q = tets + 4 * star[s];
      const double qv = 0.25 * tet_volume(pos, q);
      for (int k = 0; k < 4; ++k)
        if (new_of_old[(size_t)q[k]] >= 0) out->volume[new_of_old[(size_t)q[k]]] -= qv;
    }
    for (int64_t t = 0; t < nnew; ++t) {
      const double qv = 0.25 * tet_volume(pos, &new_tets[4 * t]);
      for (int k = 0; k < 4; ++k) out->volume[new_of_old[(size_t)new_tets[4 * t + k]]] += qv;
    }
    // tetrahedra: the untouched ones (threads over ranges, each writing at
    // the count of untouched ones before its range), then the new ones,
    // renumbered
    {
      const unsigned nt = pass_threads(ntet);
      std::vector<int64_t> base(nt + 1, 0);
      run_threads(nt, [&](unsigned th) {
        int64_t c = 0;
        for (int64_t t = range_start(ntet, th, nt), t1 = range_start(ntet, th + 1, nt); t < t1; ++t)
          c += !tet_hit[(size_t)t];
        base[th + 1] = c;
      });
      for (unsigned th = 0; th < nt; ++th) base[th + 1] += base[th];
      run_threads(nt, [&](unsigned th) {
        int32_t *t2 = out->tets + 4 * base[th];
        for (int64_t t = range_start(ntet, th, nt), t1 = range_start(ntet, th + 1, nt); t < t1; ++t) {
          if (tet_hit[(size_t)t]) continue;
          for (int k = 0; k < 4; ++k) *t2++ = new_of_old[(size_t)tets[4 * t + k]];
        }
      });
      int32_t *t2 = out->tets + 4 * base[nt];
      for (int64_t t = 0; t < 4 * nnew; ++t) *t2++ = new_of_old[(size_t)new_tets[t]];
    }
    out->n = n2;
    out->nnz = m;
    out->ntet = ntet2;
    return SX_OK;
  } catch (const std::exception &) {  // bad_alloc, or a size beyond what a vector holds
    sx_remesh_free(out);
    return SX_ENOMEM;
  }
}

extern "C" void sx_remesh_free(sx_remesh_result *r) {
  if (!r) return;
  std::free(r->row_ptr);
  std::free(r->col);
  std::free(r->volume);
  std::free(r->tets);
  std::free(r->old_of_new);
  r->row_ptr = nullptr;
  r->col = nullptr;
  r->volume = nullptr;
  r->tets = nullptr;
  r->old_of_new = nullptr;
}
