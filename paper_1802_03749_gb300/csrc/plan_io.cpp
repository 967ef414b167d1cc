// Plan serialisation: reordering and partitioning are a one-off cost that a
// later run can reuse (Sec. 2.3.2).  Little-endian binary file, host tables
// only; a loaded plan uploads its tables on first use like a built one.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "plan_internal.h"

namespace {

constexpr char kMagic[8] = {'M', 'P', 'L', 'A', 'N', '0', '0', '3'};

struct writer {
    FILE *f;
    bool ok = true;
    void raw(const void *p, size_t n)
    {
        if (ok && n && fwrite(p, 1, n, f) != n) ok = false;
    }
    template <class T>
    void pod(const T &v)
    {
        raw(&v, sizeof(T));
    }
    template <class T>
    void vec(const std::vector<T> &v)
    {
        uint64_t n = v.size();
        pod(n);
        raw(v.data(), n * sizeof(T));
    }
};

struct reader {
    FILE *f;
    bool ok = true;
    void raw(void *p, size_t n)
    {
        if (ok && n && fread(p, 1, n, f) != n) ok = false;
    }
    template <class T>
    void pod(T &v)
    {
        raw(&v, sizeof(T));
    }
    template <class T>
    void vec(std::vector<T> &v)
    {
        uint64_t n = 0;
        pod(n);
        if (!ok || n > (1ull << 34)) {
            ok = false;
            return;
        }
        v.resize(n);
        raw(v.data(), n * sizeof(T));
    }
};

template <class IO, class Plan>
void walk(IO &io, Plan &P)
{
    io.pod(P.from_size);
    io.pod(P.opts);
    io.pod(P.nmaps);
    for (int m = 0; m < MP_MAX_MAPS; ++m) {
        io.pod(P.maps[m].to_set);
        io.pod(P.maps[m].arity);
        io.pod(P.maps[m].written);
        io.pod(P.maps[m].slot);
        io.pod(P.maps[m].to_size);
        io.vec(P.maps[m].idx);
    }
    io.pod(P.ntosets);
    io.pod(P.toset_id);
    io.pod(P.toset_size);
    io.vec(P.perm_from);
    for (int s = 0; s < MP_MAX_TOSETS; ++s) io.vec(P.perm_to[s]);
    io.pod(P.nblocks);
    io.vec(P.block_offsets);
    io.vec(P.block_color);
    io.pod(P.ncolors);
    io.vec(P.color_offsets);
    io.vec(P.thread_color);
    io.vec(P.block_ncolors);
    for (int s = 0; s < MP_MAX_TOSETS; ++s) {
        io.vec(P.fp_offsets[s]);
        io.vec(P.fp_ids[s]);
    }
    io.pod(P.gat_w);
    io.vec(P.gat_tab);
    io.pod(P.inv_map);
    io.vec(P.inv_off);
    io.vec(P.inv_idx);
    io.pod(P.lmap_stride);
    io.vec(P.lmap);
    io.vec(P.desc);
    io.pod(P.stats);
}

}  // namespace

extern "C" int mesh_plan_save(const mp_plan *P, const char *path)
{
    if (!P || !path) return MP_EINVAL;
    FILE *f = fopen(path, "wb");
    if (!f) return MP_EIO;
    writer w{f};
    w.raw(kMagic, sizeof(kMagic));
    walk(w, const_cast<mp_plan &>(*P));
    bool ok = w.ok;
    if (fclose(f) != 0) ok = false;
    return ok ? MP_OK : MP_EIO;
}

extern "C" int mesh_plan_load(const char *path, mp_plan **out)
{
    if (!path || !out) return MP_EINVAL;
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return MP_EIO;
    mp_plan *P = new (std::nothrow) mp_plan();
    if (!P) {
        fclose(f);
        return MP_ENOMEM;
    }
    reader r{f};
    char magic[8];
    r.raw(magic, sizeof(magic));
    if (!r.ok || std::memcmp(magic, kMagic, sizeof(magic)) != 0) r.ok = false;
    if (r.ok) {
        try {
            walk(r, *P);
        } catch (const std::bad_alloc &) {
            r.ok = false;
        }
    }
    fclose(f);
    // structural sanity of what was read
    bool sane = r.ok && P->nmaps >= 1 && P->nmaps <= MP_MAX_MAPS && P->ntosets >= 1 && P->ntosets <= MP_MAX_TOSETS &&
                (int64_t)P->perm_from.size() == P->from_size &&
                (int64_t)P->block_offsets.size() == (int64_t)P->nblocks + 1 &&
                (int64_t)P->color_offsets.size() == (int64_t)P->ncolors + 1;
    if (sane && P->opts.coloring == MP_COLOR_HIER)
        sane = (int64_t)P->desc.size() == P->nblocks && (int64_t)P->thread_color.size() == P->from_size &&
               (int64_t)P->lmap.size() == P->from_size * (int64_t)P->lmap_stride;
    if (!sane) {
        delete P;
        return MP_EIO;
    }
    P->dev = mp_device_tables{};
    *out = P;
    return MP_OK;
}
