// Forest files: gf_forest_save / gf_forest_load.
//
// The paper keeps its forests in memory; a file lets one build serve many processes and lets a
// forest built elsewhere (by a CPU implementation of Alg. 1) be queried here.  The file holds the
// tree structure itself (splits and leaf order), so loading needs neither the build's seed nor
// its parameters and gives back the same forest bit for bit.
//
// Layout (little-endian; every section a whole number of 4-byte words):
//   header, 128 bytes
//     0  char[8]   magic "GFFOREST"
//     8  u32       version (1)
//    12  u32       0x01020304 (byte-order mark)
//    16  i64       n
//    24  i32 x 4   d, T, leaf_size, L
//    40  u32       flags: bit 0 reflections present, bit 1 bf16 screen, bit 2 fp8 screen
//    44  i32 x 12  tuning per precision: warps[3], ctas[3], rerank_R[3], rows_in_flight[3]
//    92  u32       0
//    96  u64       payload bytes
//   104  u64 x 2   checksum s1 = sum w_i, s2 = sum (i + 1) w_i (mod 2^64), the w_i the u32 words of
//                  header bytes 0..95 followed by those of the payload
//   120  u64       0
//   payload
//     nodes  [T][2^L - 1] x (i32 split dimension, f32 split value)   (Alg. 1: one split per node)
//     perm   [T][n] i32   point ids in leaf order (leaf b holds positions [b n >> L, (b+1) n >> L))
//     U      [T][d] f32   only with flag bit 0 (Sec. 2.2)
//     X      [n][d] f32   the points
#include "gf_internal.cuh"
#include "gf_trace.cuh"

#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace {

constexpr char MAGIC[8] = {'G', 'F', 'F', 'O', 'R', 'E', 'S', 'T'};
constexpr uint32_t VERSION = 1;
constexpr uint32_t BOM = 0x01020304u;
constexpr size_t HEADER_BYTES = 128;
constexpr size_t HEADER_SUMMED = 96;  // header bytes covered by the checksum (all but its own fields)
constexpr uint32_t FLAG_U = 1u, FLAG_BF16 = 2u, FLAG_FP8 = 4u;

void put32(unsigned char *b, size_t off, uint32_t v) {
    for (int i = 0; i < 4; ++i) b[off + i] = (unsigned char)(v >> (8 * i));
}
void put64(unsigned char *b, size_t off, uint64_t v) {
    for (int i = 0; i < 8; ++i) b[off + i] = (unsigned char)(v >> (8 * i));
}
uint32_t get32(const unsigned char *b, size_t off) {
    uint32_t v = 0;
    for (int i = 0; i < 4; ++i) v |= (uint32_t)b[off + i] << (8 * i);
    return v;
}
uint64_t get64(const unsigned char *b, size_t off) {
    uint64_t v = 0;
    for (int i = 0; i < 8; ++i) v |= (uint64_t)b[off + i] << (8 * i);
    return v;
}

bool host_is_little_endian() {
    const uint32_t one = 1;
    unsigned char c;
    std::memcpy(&c, &one, 1);
    return c == 1;
}

// Position-weighted sums of u32 words (a Fletcher-style check: catches changed, dropped and
// swapped words).
struct Checksum {
    uint64_t s1 = 0, s2 = 0, words = 0;
    void add(const void *p, size_t bytes) {
        const unsigned char *b = (const unsigned char *)p;
        for (size_t i = 0; i + 4 <= bytes; i += 4) {
            uint32_t w;
            std::memcpy(&w, b + i, 4);
            ++words;
            s1 += w;
            s2 += words * (uint64_t)w;
        }
    }
};

int io_fail(const char *what, const std::string &path) {
    return gf_fail(GF_EIO, "%s '%s': %s", what, path.c_str(), errno ? std::strerror(errno) : "bad file");
}

struct Writer {
    FILE *f = nullptr;
    Checksum ck;
    bool write(const void *p, size_t bytes) {
        ck.add(p, bytes);
        return bytes == 0 || std::fwrite(p, 1, bytes, f) == bytes;
    }
};

struct Reader {
    FILE *f = nullptr;
    Checksum ck;
    bool read(void *p, size_t bytes) {
        if (bytes && std::fread(p, 1, bytes, f) != bytes) return false;
        ck.add(p, bytes);
        return true;
    }
};

bool tuning_ok(const int32_t w[3], const int32_t c[3], const int32_t r[3], const int32_t g[3]) {
    for (int p = 0; p < 3; ++p)
        if (w[p] < 1 || w[p] > 32 || c[p] < 0 || c[p] > GF_MAX_CTAS_PER_SM || r[p] < 0 || r[p] > GF_MAX_SHORTLIST ||
            (g[p] != 0 && g[p] != 2 && g[p] != 4))
            return false;
    return true;
}

int save_impl(const gf_forest *F, const std::string &path) {
    const size_t nn = ((size_t)1 << F->L) - 1;
    const size_t n = (size_t)F->n, d = (size_t)F->d, T = (size_t)F->T;
    std::vector<int2> nodes(T * nn);
    std::vector<int32_t> perm(T * n);
    std::vector<float> U(F->U ? T * d : 0);
    GF_CUDA_TRY(cudaDeviceSynchronize());
    if (!nodes.empty())  // a single-leaf forest (L = 0) has no internal node
        GF_CUDA_TRY(cudaMemcpy(nodes.data(), F->nodes, nodes.size() * sizeof(int2), cudaMemcpyDeviceToHost));
    GF_CUDA_TRY(cudaMemcpy(perm.data(), F->perm, perm.size() * 4, cudaMemcpyDeviceToHost));
    if (F->U) GF_CUDA_TRY(cudaMemcpy(U.data(), F->U, U.size() * 4, cudaMemcpyDeviceToHost));
    // X leaves the device in slabs of about 64 MB (rows unpadded: the file holds d floats a row).
    const size_t slab_rows = std::max<size_t>(1, ((size_t)64 << 20) / (d * 4));
    std::vector<float> slab(std::min(slab_rows, n) * d);

    const std::string tmp = path + ".tmp";
    Writer w;
    errno = 0;
    w.f = std::fopen(tmp.c_str(), "wb");
    if (!w.f) return io_fail("cannot create", tmp);
    unsigned char hdr[HEADER_BYTES] = {};
    std::memcpy(hdr, MAGIC, 8);
    put32(hdr, 8, VERSION);
    put32(hdr, 12, BOM);
    put64(hdr, 16, (uint64_t)F->n);
    put32(hdr, 24, (uint32_t)F->d);
    put32(hdr, 28, (uint32_t)F->T);
    put32(hdr, 32, (uint32_t)F->leaf_size);
    put32(hdr, 36, (uint32_t)F->L);
    put32(hdr, 40, (F->U ? FLAG_U : 0) | (F->xb ? FLAG_BF16 : 0) | (F->x8 ? FLAG_FP8 : 0));
    for (int p = 0; p < 3; ++p) {
        put32(hdr, 44 + 4 * p, (uint32_t)F->tune_warps[p]);
        put32(hdr, 56 + 4 * p, (uint32_t)F->tune_ctas[p]);
        put32(hdr, 68 + 4 * p, (uint32_t)F->tune_R[p]);
        put32(hdr, 80 + 4 * p, (uint32_t)F->tune_G[p]);
    }
    bool ok = std::fwrite(hdr, 1, HEADER_BYTES, w.f) == HEADER_BYTES;
    w.ck = Checksum();
    w.ck.add(hdr, HEADER_SUMMED);  // the header's fields, then the payload
    ok = ok && w.write(nodes.data(), nodes.size() * sizeof(int2));
    ok = ok && w.write(perm.data(), perm.size() * 4);
    ok = ok && w.write(U.data(), U.size() * 4);
    for (size_t r0 = 0; ok && r0 < n; r0 += slab_rows) {
        const size_t rows = std::min(slab_rows, n - r0);
        cudaError_t e = cudaMemcpy2D(slab.data(), d * 4, F->x + r0 * F->ldx, (size_t)F->ldx * 4, d * 4, rows,
                                     cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            std::fclose(w.f);
            std::remove(tmp.c_str());
            return gf_cuda_fail(e, "copy X to the host");
        }
        ok = w.write(slab.data(), rows * d * 4);
    }
    if (ok) {
        put64(hdr, 96, w.ck.words * 4 - HEADER_SUMMED);
        put64(hdr, 104, w.ck.s1);
        put64(hdr, 112, w.ck.s2);
        ok = std::fseek(w.f, 0, SEEK_SET) == 0 && std::fwrite(hdr, 1, HEADER_BYTES, w.f) == HEADER_BYTES &&
             std::fflush(w.f) == 0;
    }
    const int saved_errno = errno;
    ok = (std::fclose(w.f) == 0) && ok;
    if (!ok) {
        std::remove(tmp.c_str());
        errno = saved_errno;
        return io_fail("cannot write", tmp);
    }
    // The new file replaces an old one only once it is complete.
    errno = 0;
    if (std::rename(tmp.c_str(), path.c_str()) != 0) {
        const int e = errno;
        std::remove(tmp.c_str());
        errno = e;
        return io_fail("cannot rename to", path);
    }
    return GF_OK;
}

int load_impl(const std::string &path, gf_forest **out) {
    Reader rd;
    errno = 0;
    rd.f = std::fopen(path.c_str(), "rb");
    if (!rd.f) return io_fail("cannot open", path);
    struct Closer {
        FILE *f;
        ~Closer() { std::fclose(f); }
    } closer{rd.f};

    unsigned char hdr[HEADER_BYTES];
    errno = 0;
    if (std::fread(hdr, 1, HEADER_BYTES, rd.f) != HEADER_BYTES) return io_fail("short header in", path);
    if (std::memcmp(hdr, MAGIC, 8) != 0) return gf_fail(GF_EIO, "'%s' is not a forest file", path.c_str());
    if (get32(hdr, 8) != VERSION) return gf_fail(GF_EIO, "'%s': unsupported version %u", path.c_str(), get32(hdr, 8));
    if (get32(hdr, 12) != BOM) return gf_fail(GF_EIO, "'%s': bad byte-order mark", path.c_str());
    const int64_t n = (int64_t)get64(hdr, 16);
    const int32_t d = (int32_t)get32(hdr, 24), T = (int32_t)get32(hdr, 28);
    const int32_t leaf_size = (int32_t)get32(hdr, 32), L = (int32_t)get32(hdr, 36);
    const uint32_t flags = get32(hdr, 40);
    int32_t tw[3], tc[3], tr[3], tg[3];
    for (int p = 0; p < 3; ++p) {
        tw[p] = (int32_t)get32(hdr, 44 + 4 * p);
        tc[p] = (int32_t)get32(hdr, 56 + 4 * p);
        tr[p] = (int32_t)get32(hdr, 68 + 4 * p);
        tg[p] = (int32_t)get32(hdr, 80 + 4 * p);
    }
    if (n < 1 || n > 0x7fffffffLL || d < 1 || d > 65535 || T < 1 || T > 4096 || leaf_size < 1 ||
        L != depth_of(n, leaf_size) || L > 30 || (flags & ~(FLAG_U | FLAG_BF16 | FLAG_FP8)) != 0 ||
        get32(hdr, 92) != 0 || get64(hdr, 120) != 0 || !tuning_ok(tw, tc, tr, tg))
        return gf_fail(GF_EIO, "'%s': bad header", path.c_str());
    const size_t nn = ((size_t)1 << L) - 1;
    const uint64_t expect = (uint64_t)T * nn * 8 + (uint64_t)T * n * 4 + ((flags & FLAG_U) ? (uint64_t)T * d * 4 : 0) +
                            (uint64_t)n * d * 4;
    if (get64(hdr, 96) != expect)
        return gf_fail(GF_EIO, "'%s': payload of %llu bytes, the header's sizes give %llu", path.c_str(),
                       (unsigned long long)get64(hdr, 96), (unsigned long long)expect);
    if (std::fseek(rd.f, 0, SEEK_END) != 0) return io_fail("cannot seek in", path);
    const long long size = std::ftell(rd.f);
    if (size < 0 || (uint64_t)size != HEADER_BYTES + expect)
        return gf_fail(GF_EIO, "'%s': %lld bytes, expected %llu (truncated or trailing data)", path.c_str(), size,
                       (unsigned long long)(HEADER_BYTES + expect));
    if (std::fseek(rd.f, (long)HEADER_BYTES, SEEK_SET) != 0) return io_fail("cannot seek in", path);
    rd.ck.add(hdr, HEADER_SUMMED);

    std::vector<int2> nodes((size_t)T * nn);
    std::vector<int32_t> perm((size_t)T * n);
    std::vector<float> U((flags & FLAG_U) ? (size_t)T * d : 0);
    std::vector<float> X((size_t)n * d);
    errno = 0;
    if (!rd.read(nodes.data(), nodes.size() * sizeof(int2)) || !rd.read(perm.data(), perm.size() * 4) ||
        !rd.read(U.data(), U.size() * 4) || !rd.read(X.data(), X.size() * 4))
        return io_fail("short read of", path);
    if (rd.ck.s1 != get64(hdr, 104) || rd.ck.s2 != get64(hdr, 112))
        return gf_fail(GF_EIO, "'%s': checksum mismatch (the file is damaged)", path.c_str());
    std::vector<int32_t> split_dim(nodes.size());
    std::vector<float> split_val(nodes.size());
    for (size_t i = 0; i < nodes.size(); ++i) {
        split_dim[i] = nodes[i].x;
        std::memcpy(&split_val[i], &nodes[i].y, 4);
    }
    for (float u : U)
        if (!std::isfinite(u)) return gf_fail(GF_EIO, "'%s': reflections hold NaN/Inf", path.c_str());

    // Everything above ran on the host; the device is touched from here on.
    gf_forest *F = nullptr;
    int r = gf_forest_alloc(&F, X.data(), n, d, T, leaf_size, false, 0);
    if (r) return r;
    r = gf_forest_fill_structure(F, split_dim.data(), split_val.data(), perm.data());
    if (r == GF_EINVAL) {
        const std::string why = gf_last_error();
        r = gf_fail(GF_EIO, "'%s' holds an invalid forest: %s", path.c_str(), why.c_str());
    }
    if (!r && (flags & FLAG_U)) r = gf_forest_set_U(F, U.data());
    if (!r && (flags & FLAG_BF16)) r = gf_forest_add_screen(F, GF_BF16_RERANK, nullptr);
    if (!r && (flags & FLAG_FP8)) r = gf_forest_add_screen(F, GF_FP8_RERANK, nullptr);
    if (r) {
        gf_forest_destroy(F);
        return r;
    }
    for (int p = 0; p < 3; ++p) {
        F->tune_warps[p] = tw[p];
        F->tune_ctas[p] = tc[p];
        F->tune_R[p] = tr[p];
        F->tune_G[p] = tg[p];
    }
    *out = F;
    return GF_OK;
}

}  // namespace

extern "C" int gf_forest_save(const gf_forest *F, const char *path) {
    GfRange range("gf_forest_save");
    if (!F || !path || !*path) return gf_fail(GF_EINVAL, "null forest or empty path");
    if (!host_is_little_endian()) return gf_fail(GF_EUNSUPPORTED, "forest files need a little-endian host");
    try {
        return save_impl(F, path);
    } catch (const std::bad_alloc &) {
        return gf_fail(GF_ENOMEM, "host allocation failed while saving '%s'", path);
    }
}

extern "C" int gf_forest_load(const char *path, gf_forest **out) {
    GfRange range("gf_forest_load");
    if (!out) return gf_fail(GF_EINVAL, "out is null");
    *out = nullptr;
    if (!path || !*path) return gf_fail(GF_EINVAL, "empty path");
    if (!host_is_little_endian()) return gf_fail(GF_EUNSUPPORTED, "forest files need a little-endian host");
    try {
        return load_impl(path, out);
    } catch (const std::bad_alloc &) {
        return gf_fail(GF_ENOMEM, "host allocation failed while loading '%s'", path);
    }
}
