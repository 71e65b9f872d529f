// Writes a checkpoint-shaped file through the checkpoint writer of the
// library (sx_ckpt_io.h): the checkpoint magic, then pseudo-random bytes in
// writes of the sizes given on the command line, then the checksum trailer;
// and checks it back with the library's verification.  Built and run by
// test_checkpoint_file.py.
//   ckpt_driver <path> <seed> <size>...
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "sx_ckpt_io.h"

int main(int argc, char **argv) {
  if (argc < 4) return 2;
  static const char kMagic[8] = {'S', 'X', 'C', 'K', 'P', 'T', '0', '3'};
  uint64_t state = std::strtoull(argv[2], nullptr, 10) * 2 + 1;
  {
    sx::File f(argv[1], "wb");
    if (!f.f || !f.write(kMagic, 8)) return 3;
    for (int a = 3; a < argc; ++a) {
      std::vector<unsigned char> b(std::strtoull(argv[a], nullptr, 10));
      for (unsigned char &c : b) {
        state = state * 6364136223846793005ull + 1442695040888963407ull;
        c = (unsigned char)(state >> 56);
      }
      if (!f.write(b.data(), b.size())) return 3;
    }
    if (!sx::write_trailer(f)) return 3;
  }
  std::string why;
  if (!sx::verify_checkpoint_file(argv[1], kMagic, why)) {
    std::fprintf(stderr, "%s\n", why.c_str());
    return 4;
  }
  return 0;
}
