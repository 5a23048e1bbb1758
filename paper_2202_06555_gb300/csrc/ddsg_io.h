// ddsg_io.h -- the pieces of libddsg's checkpoint files: a byte buffer writer and
// a bounds-checked reader, FNV-1a checksums, whole-file read and write. Every file
// is an 8-byte magic, a u32 version, a u32 0, the body, and the u64 FNV-1a of
// the body (all bytes after the 16-byte header), little-endian host layout.
#pragma once
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <vector>

namespace ddsg {
namespace io {

inline uint64_t fnv1a(const unsigned char *p, size_t n, uint64_t hsh = 0xcbf29ce484222325ull) {
    for (size_t i = 0; i < n; ++i) {
        hsh ^= p[i];
        hsh *= 0x100000001b3ull;
    }
    return hsh;
}

struct Writer {
    std::vector<unsigned char> buf;
    template <typename T>
    void put(const T *v, size_t n) {
        const unsigned char *b = reinterpret_cast<const unsigned char *>(v);
        buf.insert(buf.end(), b, b + sizeof(T) * n);
    }
    template <typename T>
    void put1(T v) { put(&v, 1); }
    // magic and version; the body starts after them
    void header(const char magic[8], uint32_t version) {
        put(magic, 8);
        put1<uint32_t>(version);
        put1<uint32_t>(0);
    }
    // appends the checksum of the body
    void seal() { put1<uint64_t>(fnv1a(buf.data() + 16, buf.size() - 16)); }
};

struct Reader {
    const unsigned char *p, *end;
    bool ok = true;
    template <typename T>
    bool get(T *v, size_t n) {
        const size_t b = sizeof(T) * n;
        if (!ok || (size_t)(end - p) < b) return ok = false;
        memcpy(v, p, b);
        p += b;
        return true;
    }
};

inline bool write_file(const char *path, const std::vector<unsigned char> &buf) {
    FILE *f = fopen(path, "wb");
    if (!f) return false;
    const size_t wr = fwrite(buf.data(), 1, buf.size(), f);
    const int cl = fclose(f);
    return wr == buf.size() && cl == 0;
}

inline bool read_file(const char *path, std::vector<unsigned char> &buf) {
    FILE *f = fopen(path, "rb");
    if (!f) return false;
    buf.clear();
    unsigned char chunk[1 << 16];
    size_t got;
    while ((got = fread(chunk, 1, sizeof chunk, f)) > 0) buf.insert(buf.end(), chunk, chunk + got);
    fclose(f);
    return true;
}

// Checks magic, version and checksum; on success a Reader over the body.
// Returns 0, or 1 wrong magic / too short, 2 wrong version, 3 checksum mismatch.
inline int open_body(const std::vector<unsigned char> &buf, const char magic[8], uint32_t version, Reader &r,
                     uint32_t *found_version = nullptr) {
    if (buf.size() < 16 + 8 || memcmp(buf.data(), magic, 8) != 0) return 1;
    uint32_t v = 0;
    memcpy(&v, buf.data() + 8, 4);
    if (found_version) *found_version = v;
    if (v != version) return 2;
    uint64_t sum = 0;
    memcpy(&sum, buf.data() + buf.size() - 8, 8);
    if (fnv1a(buf.data() + 16, buf.size() - 16 - 8) != sum) return 3;
    r = Reader{buf.data() + 16, buf.data() + buf.size() - 8};
    return 0;
}

}  // namespace io
}  // namespace ddsg
