// Checkpoint / resume of a lattice handle.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "common.cuh"

namespace hp {
namespace {

uint32_t crc32_update(uint32_t crc, const unsigned char* p, size_t n) {
    // reflected CRC-32 (polynomial 0xEDB88320), bitwise
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) {
        crc ^= p[i];
        for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
    }
    return ~crc;
}

struct CkptHeader {
    char magic[8];      // "HPCKPT1\0"
    hp_desc desc;
    uint64_t sweep;
    int32_t has_mp;
    int32_t pad;
    uint64_t n;         // sites
};

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" int hp_checkpoint_save(hp_handle* h, const char* path, void* stream) {
    if (!h || !path) return set_error(HP_ERR_ARG, "hp_checkpoint_save: null argument");
    if (!h->q) return set_error(HP_ERR_STATE, "hp_checkpoint_save: no lattice bound");
    cudaStream_t s = as_stream(stream);
    const size_t n = (size_t)h->lat.N;
    std::vector<int32_t> q(n), mp(h->mp ? n : 0);
    HP_CUDA(cudaMemcpyAsync(q.data(), h->q, n * 4, cudaMemcpyDeviceToHost, s));
    if (h->mp) HP_CUDA(cudaMemcpyAsync(mp.data(), h->mp, n * 4, cudaMemcpyDeviceToHost, s));
    HP_CUDA(cudaStreamSynchronize(s));
    CkptHeader hd;
    memset(&hd, 0, sizeof hd);
    memcpy(hd.magic, "HPCKPT1", 8);
    hd.desc = h->desc;
    hd.sweep = h->sweep;
    hd.has_mp = h->mp != nullptr;
    hd.n = n;
    uint32_t crc = crc32_update(0, reinterpret_cast<const unsigned char*>(&hd), sizeof hd);
    crc = crc32_update(crc, reinterpret_cast<const unsigned char*>(q.data()), n * 4);
    if (h->mp) crc = crc32_update(crc, reinterpret_cast<const unsigned char*>(mp.data()), n * 4);
    FILE* f = fopen(path, "wb");
    if (!f) return set_error(HP_ERR_ARG, std::string("hp_checkpoint_save: cannot open ") + path);
    bool ok = fwrite(&hd, sizeof hd, 1, f) == 1 && fwrite(q.data(), 4, n, f) == n &&
              (!h->mp || fwrite(mp.data(), 4, n, f) == n) && fwrite(&crc, 4, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    return ok ? HP_OK : set_error(HP_ERR_ARG, "hp_checkpoint_save: write failed");
}

extern "C" int hp_checkpoint_load(hp_handle* h, const char* path, void* stream) {
    if (!h || !path) return set_error(HP_ERR_ARG, "hp_checkpoint_load: null argument");
    if (!h->q) return set_error(HP_ERR_STATE, "hp_checkpoint_load: no lattice bound");
    FILE* f = fopen(path, "rb");
    if (!f) return set_error(HP_ERR_ARG, std::string("hp_checkpoint_load: cannot open ") + path);
    CkptHeader hd;
    const size_t n = (size_t)h->lat.N;
    std::vector<int32_t> q, mp;
    uint32_t crc_file = 0;
    bool ok = fread(&hd, sizeof hd, 1, f) == 1 && memcmp(hd.magic, "HPCKPT1", 8) == 0;
    if (ok && (hd.n != n || memcmp(&hd.desc, &h->desc, sizeof hd.desc) != 0 || (hd.has_mp != 0) != (h->mp != nullptr))) {
        fclose(f);
        return set_error(HP_ERR_ARG, "hp_checkpoint_load: checkpoint belongs to a different lattice");
    }
    if (ok) {
        q.resize(n);
        ok = fread(q.data(), 4, n, f) == n;
        if (ok && hd.has_mp) { mp.resize(n); ok = fread(mp.data(), 4, n, f) == n; }
        ok = ok && fread(&crc_file, 4, 1, f) == 1;
    }
    fclose(f);
    if (!ok) return set_error(HP_ERR_CHECKSUM, "hp_checkpoint_load: truncated or not a checkpoint");
    uint32_t crc = crc32_update(0, reinterpret_cast<const unsigned char*>(&hd), sizeof hd);
    crc = crc32_update(crc, reinterpret_cast<const unsigned char*>(q.data()), n * 4);
    if (hd.has_mp) crc = crc32_update(crc, reinterpret_cast<const unsigned char*>(mp.data()), n * 4);
    if (crc != crc_file) return set_error(HP_ERR_CHECKSUM, "hp_checkpoint_load: checksum mismatch");
    cudaStream_t s = as_stream(stream);
    HP_CUDA(cudaMemcpyAsync(h->q, q.data(), n * 4, cudaMemcpyHostToDevice, s));
    if (hd.has_mp) HP_CUDA(cudaMemcpyAsync(h->mp, mp.data(), n * 4, cudaMemcpyHostToDevice, s));
    HP_CUDA(cudaStreamSynchronize(s));
    h->sweep = hd.sweep;
    return HP_OK;
}
