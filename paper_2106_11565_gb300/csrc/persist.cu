// Save and load of a built index (flinng_save / flinng_load, declared in
// include/flinng.h). The file holds the configuration, the hash parameters
// and every array a query reads: group ids, member lists and records, the
// CSR of each table and the heavy slots' cell bitmaps. Build scratch is not
// saved. A loaded index answers every query as the saved one did, and takes
// inserts up to the same capacity.
//
// Layout (little endian, as written by this library on the same kind of
// host): Header, then the parameters (cosine: P x dim fp32 projections;
// Jaccard: P uint64 multipliers and L uint64 offsets), then gid (n x rp
// uint16), moff (B*R + 1 uint32), mem (R*n uint32), mrec (n x rw uint32),
// off and hidx (L*2^W + 1 uint32 each), cells (n_cells uint16) and the
// heavy bitmaps (n_heavy x ceil(B*R/32) uint32).
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "trace.h"

using namespace flinng;

namespace {

constexpr char kMagic[8] = {'F', 'L', 'I', 'N', 'N', 'G', 'I', 'X'};
constexpr uint32_t kVersion = 1;

struct Header {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    flinng_config cfg;
    uint32_t doph_a, doph_b;
    uint64_t doph_seed;
    uint64_t n_points, n_cells;
    uint32_t n_heavy, pad;
};

struct File {
    FILE *f = nullptr;
    ~File() { if (f) fclose(f); }
};

template <class T>
int dump(FILE *f, const T *dev, uint64_t n, cudaStream_t st, std::vector<unsigned char> &buf)
{
    if (n == 0) return FLINNG_OK;
    buf.resize(n * sizeof(T));
    FL_CUDA(cudaMemcpyAsync(buf.data(), dev, n * sizeof(T), cudaMemcpyDeviceToHost, st));
    FL_CUDA(cudaStreamSynchronize(st));
    if (fwrite(buf.data(), sizeof(T), n, f) != n) return set_error(FLINNG_ERR_INVALID_ARG, "save: write failed");
    return FLINNG_OK;
}

template <class T>
int undump(FILE *f, T *dev, uint64_t n, cudaStream_t st, std::vector<unsigned char> &buf)
{
    if (n == 0) return FLINNG_OK;
    buf.resize(n * sizeof(T));
    if (fread(buf.data(), sizeof(T), n, f) != n) return set_error(FLINNG_ERR_INVALID_ARG, "load: file too short");
    FL_CUDA(cudaMemcpyAsync(dev, buf.data(), n * sizeof(T), cudaMemcpyHostToDevice, st));
    FL_CUDA(cudaStreamSynchronize(st));
    return FLINNG_OK;
}

template <class T>
int read_host(FILE *f, std::vector<T> &v, uint64_t n)
{
    v.resize(n);
    if (n && fread(v.data(), sizeof(T), n, f) != n) return set_error(FLINNG_ERR_INVALID_ARG, "load: file too short");
    return FLINNG_OK;
}

}  // namespace

extern "C" int flinng_save(flinng_index *idx, const char *path)
{
    TraceRange trace_("flinng_save");
    if (!idx || !path) return set_error(FLINNG_ERR_INVALID_ARG, "save: null argument");
    const cudaStream_t st = idx->stream;
    FL_CUDA(cudaStreamSynchronize(st));
    File fh;
    fh.f = fopen(path, "wb");
    if (!fh.f) return set_error(FLINNG_ERR_INVALID_ARG, "save: cannot open %s", path);
    Header h{};
    std::memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.header_bytes = sizeof(Header);
    h.cfg = idx->cfg;
    h.doph_a = idx->doph_a;
    h.doph_b = idx->doph_b;
    h.doph_seed = idx->doph_seed;
    h.n_points = idx->n_points;
    h.n_cells = idx->n_cells;
    h.n_heavy = idx->n_heavy;
    if (fwrite(&h, sizeof h, 1, fh.f) != 1) return set_error(FLINNG_ERR_INVALID_ARG, "save: write failed");
    std::vector<unsigned char> buf;
    const uint64_t n = idx->n_points;
    if (idx->cfg.metric == FLINNG_COSINE_SRP) {
        FL_TRY(dump(fh.f, idx->srp_w, uint64_t(idx->P) * idx->cfg.dim, st, buf));
    } else {
        FL_TRY(dump(fh.f, idx->bucket_a, uint64_t(idx->P), st, buf));
        FL_TRY(dump(fh.f, idx->bucket_c, uint64_t(idx->cfg.L), st, buf));
    }
    FL_TRY(dump(fh.f, idx->gid, n * idx->rp, st, buf));
    FL_TRY(dump(fh.f, idx->moff, uint64_t(idx->BR) + 1, st, buf));
    FL_TRY(dump(fh.f, idx->mem, uint64_t(idx->cfg.R) * n, st, buf));
    FL_TRY(dump(fh.f, idx->mrec, n * idx->rw, st, buf));
    FL_TRY(dump(fh.f, idx->off, idx->nslot + 1, st, buf));
    FL_TRY(dump(fh.f, idx->hidx, idx->nslot + 1, st, buf));
    FL_TRY(dump(fh.f, idx->cells, idx->n_cells, st, buf));
    FL_TRY(dump(fh.f, idx->hbm, uint64_t(idx->n_heavy) * idx->BRw, st, buf));
    if (fflush(fh.f) != 0) return set_error(FLINNG_ERR_INVALID_ARG, "save: write failed");
    return FLINNG_OK;
}

extern "C" int flinng_load(const char *path, void *stream, flinng_index **out)
{
    TraceRange trace_("flinng_load");
    if (!path || !out) return set_error(FLINNG_ERR_INVALID_ARG, "load: null argument");
    *out = nullptr;
    File fh;
    fh.f = fopen(path, "rb");
    if (!fh.f) return set_error(FLINNG_ERR_INVALID_ARG, "load: cannot open %s", path);
    Header h{};
    if (fread(&h, sizeof h, 1, fh.f) != 1 || std::memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion ||
        h.header_bytes != sizeof(Header))
        return set_error(FLINNG_ERR_INVALID_ARG, "load: %s is not an index file of this version", path);
    const flinng_config &cfg = h.cfg;
    flinng_params p{};
    std::vector<float> w;
    std::vector<uint64_t> ba, bc;
    const uint64_t P = uint64_t(cfg.L) * cfg.K;
    if (cfg.metric == FLINNG_COSINE_SRP) {
        if (P * cfg.dim > (uint64_t(1) << 34)) return set_error(FLINNG_ERR_INVALID_ARG, "load: bad header");
        FL_TRY(read_host(fh.f, w, P * cfg.dim));
        p.srp_w = w.data();
    } else {
        if (P > (uint64_t(1) << 24)) return set_error(FLINNG_ERR_INVALID_ARG, "load: bad header");
        FL_TRY(read_host(fh.f, ba, P));
        FL_TRY(read_host(fh.f, bc, cfg.L));
        p.doph_a = h.doph_a;
        p.doph_b = h.doph_b;
        p.doph_seed = h.doph_seed;
        p.bucket_a = ba.data();
        p.bucket_c = bc.data();
    }
    flinng_index *ix = nullptr;
    FL_TRY(flinng_create(&cfg, &p, stream, &ix));   // checks the configuration, allocates by capacity
    int rc = FLINNG_OK;
    if (h.n_points > cfg.capacity || h.n_cells > ix->entries_cap)
        rc = set_error(FLINNG_ERR_INVALID_ARG, "load: %s holds more than its capacity", path);
    const cudaStream_t st = ix->stream;
    std::vector<unsigned char> buf;
    const uint64_t n = h.n_points;
    if (rc == FLINNG_OK && h.n_heavy > 0) {
        const uint64_t words = uint64_t(h.n_heavy) * ix->BRw;
        const cudaError_t e = cudaMalloc(&ix->hbm, words * 4);
        if (e != cudaSuccess) {
            rc = cuda_error(e, "load: cell bitmaps");
        } else {
            ix->hbm_words = words;
            ix->device_bytes += words * 4;
        }
    }
    if (rc == FLINNG_OK) rc = undump(fh.f, ix->gid, n * ix->rp, st, buf);
    if (rc == FLINNG_OK) rc = undump(fh.f, ix->moff, uint64_t(ix->BR) + 1, st, buf);
    if (rc == FLINNG_OK) rc = undump(fh.f, ix->mem, uint64_t(cfg.R) * n, st, buf);
    if (rc == FLINNG_OK) rc = undump(fh.f, ix->mrec, n * ix->rw, st, buf);
    if (rc == FLINNG_OK) rc = undump(fh.f, ix->off, ix->nslot + 1, st, buf);
    if (rc == FLINNG_OK) rc = undump(fh.f, ix->hidx, ix->nslot + 1, st, buf);
    if (rc == FLINNG_OK) rc = undump(fh.f, ix->cells, h.n_cells, st, buf);
    if (rc == FLINNG_OK) rc = undump(fh.f, ix->hbm, uint64_t(h.n_heavy) * ix->BRw, st, buf);
    if (rc != FLINNG_OK) {
        flinng_destroy(ix);
        return rc;
    }
    ix->n_points = n;
    ix->n_cells = h.n_cells;
    ix->n_heavy = h.n_heavy;
    *out = ix;
    return FLINNG_OK;
}

extern "C" int flinng_get_config(const flinng_index *idx, flinng_config *out)
{
    if (!idx || !out) return set_error(FLINNG_ERR_INVALID_ARG, "get_config: null argument");
    *out = idx->cfg;
    return FLINNG_OK;
}
