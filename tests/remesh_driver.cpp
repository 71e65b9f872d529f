// Stand-alone driver for sx_remesh_remove, built with a sanitizer by
// test_remesh_sanitizers.py: reads a grid and the removed vertices from raw
// files in the directory given as argv[1], removes them, and writes the new
// grid beside them.  A malformed tetrahedron list must be refused.
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "simplexgb.h"

template <class T>
static std::vector<T> load(const std::string &f) {
  std::vector<T> v;
  if (FILE *fp = std::fopen(f.c_str(), "rb")) {
    T x;
    while (std::fread(&x, sizeof(T), 1, fp) == 1) v.push_back(x);
    std::fclose(fp);
  }
  return v;
}

template <class T>
static void save(const std::string &f, const T *p, int64_t n) {
  FILE *fp = std::fopen(f.c_str(), "wb");
  std::fwrite(p, sizeof(T), (size_t)n, fp);
  std::fclose(fp);
}

int main(int argc, char **argv) {
  if (argc != 2) return 2;
  const std::string d = std::string(argv[1]) + "/";
  const auto hdr = load<int64_t>(d + "hdr");  // n, ntet, nrem
  if (hdr.size() != 3) return 2;
  const auto pos = load<double>(d + "pos");
  const auto rp = load<int64_t>(d + "row_ptr");
  const auto col = load<int32_t>(d + "col");
  auto tets = load<int32_t>(d + "tets");
  const auto vol = load<double>(d + "volume");
  const auto rem = load<int32_t>(d + "removed");
  sx_remesh_result r;
  int rc = sx_remesh_remove(hdr[0], pos.data(), rp.data(), col.data(), hdr[1], tets.data(), vol.data(),
                            hdr[2], rem.data(), &r);
  if (rc != SX_OK) return 3;
  save(d + "out_hdr", &r.n, 3);
  save(d + "out_row_ptr", r.row_ptr, r.n + 1);
  save(d + "out_col", r.col, r.nnz);
  save(d + "out_volume", r.volume, r.n);
  save(d + "out_tets", r.tets, 4 * r.ntet);
  save(d + "out_old_of_new", r.old_of_new, r.n);
  sx_remesh_free(&r);
  tets[4 * (hdr[1] / 2) + 1] = (int32_t)hdr[0];
  rc = sx_remesh_remove(hdr[0], pos.data(), rp.data(), col.data(), hdr[1], tets.data(), vol.data(),
                        hdr[2], rem.data(), &r);
  return rc == SX_EINVAL && r.row_ptr == nullptr ? 0 : 4;
}
