// sx_ckpt_io.h -- host-side file handling of checkpoints: a file whose
// writes are checksummed, the checksum trailer, and the check of a file
// against its trailer.  Plain C++ (no CUDA), so that the same code can be
// built and tested on a host without a GPU.
//
// A checkpoint is the byte stream sx_save writes (header, bins, sources,
// workspace regions) followed by a 16-byte trailer: an 8-byte magic and the
// checksum of every byte before it.
#pragma once

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <sys/types.h>
#include <unistd.h>
#include <vector>

namespace sx {

// Eight FNV-1a (64-bit) streams, the byte at offset i going to stream i mod 8,
// folded together with the byte count.  The value depends only on the bytes
// and their offsets, not on how the stream is cut into calls.  Each stream
// step (xor with a byte, multiply by an odd constant) is a bijection of the
// state, so changing any one byte always changes the result.
struct ByteHash {
  static constexpr uint64_t kBasis = 0xcbf29ce484222325ull;
  static constexpr uint64_t kPrime = 0x100000001b3ull;
  uint64_t lane[8];
  uint64_t count = 0;

  ByteHash() {
    for (uint64_t &l : lane) l = kBasis;
  }
  void update(const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    size_t i = 0;
    for (; i < n && ((count + i) & 7); ++i) lane[(count + i) & 7] = (lane[(count + i) & 7] ^ b[i]) * kPrime;
    for (; i + 8 <= n; i += 8)  // here count + i is a multiple of 8
      for (int k = 0; k < 8; ++k) lane[k] = (lane[k] ^ b[i + k]) * kPrime;
    for (; i < n; ++i) lane[(count + i) & 7] = (lane[(count + i) & 7] ^ b[i]) * kPrime;
    count += n;
  }
  uint64_t digest() const {
    uint64_t h = kBasis;
    for (uint64_t l : lane) h = (h ^ l) * kPrime;
    return (h ^ count) * kPrime;
  }
};

// A file opened with fopen; every byte written through write() is hashed.
struct File {
  FILE *f = nullptr;
  ByteHash hash;
  explicit File(const char *path, const char *mode) : f(std::fopen(path, mode)) {}
  File(const File &) = delete;
  File &operator=(const File &) = delete;
  ~File() {
    if (f) std::fclose(f);
  }
  bool write(const void *p, size_t n) {
    if (n == 0) return true;
    hash.update(p, n);
    return std::fwrite(p, 1, n, f) == n;
  }
  bool read(void *p, size_t n) { return n == 0 || std::fread(p, 1, n, f) == n; }
  bool close() {  // true if the file closed cleanly
    if (!f) return false;
    const int r = std::fclose(f);
    f = nullptr;
    return r == 0;
  }
};

constexpr char kCkptSumMagic[8] = {'S', 'X', 'C', 'K', 'S', 'U', 'M', '1'};
struct CkptTrailer {
  char magic[8];
  uint64_t checksum;  // ByteHash of every byte before the trailer
};
static_assert(sizeof(CkptTrailer) == 16, "trailer layout");

// Ends a file written through f: appends the trailer (not hashed), flushes
// it and asks the system to put it on storage (fsync).
inline bool write_trailer(File &f) {
  CkptTrailer t;
  std::memcpy(t.magic, kCkptSumMagic, 8);
  t.checksum = f.hash.digest();
  return std::fwrite(&t, 1, sizeof(t), f.f) == sizeof(t) && std::fflush(f.f) == 0 &&
         fsync(fileno(f.f)) == 0;
}

// Reads the open file f through from its start and checks that it starts
// with magic (8 bytes) and ends with a trailer whose checksum matches the
// bytes before it.  Returns true, or false with the reason in why; the file
// position is left anywhere (seek before reading on).
inline bool verify_checkpoint_stream(File &f, const char magic[8], std::string &why) {
  if (!f.f) {
    why = "cannot open";
    return false;
  }
  if (fseeko(f.f, 0, SEEK_END) != 0) {
    why = "cannot seek";
    return false;
  }
  const off_t size = ftello(f.f);
  if (size < (off_t)(8 + sizeof(CkptTrailer)) || fseeko(f.f, 0, SEEK_SET) != 0) {
    why = "too short to be a checkpoint";
    return false;
  }
  std::vector<unsigned char> buf((size_t)1 << 22);
  ByteHash h;
  uint64_t left = (uint64_t)size - sizeof(CkptTrailer);
  bool first = true;
  while (left > 0) {
    const size_t k = left < buf.size() ? (size_t)left : buf.size();
    if (!f.read(buf.data(), k)) {
      why = "read failed";
      return false;
    }
    if (first && std::memcmp(buf.data(), magic, 8) != 0) {
      why = "not a checkpoint";
      return false;
    }
    first = false;
    h.update(buf.data(), k);
    left -= k;
  }
  CkptTrailer t;
  if (!f.read(&t, sizeof(t)) || std::memcmp(t.magic, kCkptSumMagic, 8) != 0) {
    why = "no checksum trailer";
    return false;
  }
  if (t.checksum != h.digest()) {
    why = "checksum mismatch: the file is damaged";
    return false;
  }
  return true;
}

// The same check of the file at path.
inline bool verify_checkpoint_file(const char *path, const char magic[8], std::string &why) {
  File f(path, "rb");
  return verify_checkpoint_stream(f, magic, why);
}

}  // namespace sx
