// Batching of many meshes into one launch per colour phase.
//
// mesh_batch_build fuses the plans of several meshes of the same loop into a
// single plan over the disjoint union of the meshes: data of mesh k sit after
// those of meshes 0..k-1 in every set (concatenated arrays, original plan
// numbering inside each mesh).  The fused block-descriptor table lists every
// mesh's blocks grouped by block colour (colour phase c holds the colour-c
// blocks of all meshes), with iteration ranges and footprint ids offset into
// the concatenation, so the staged kernels process a whole batch with one
// launch per colour phase.  Meshes keep their own block size, reordering and
// colouring; the launch uses the largest block size.
#include <algorithm>
#include <new>

#include "plan_internal.h"

extern "C" int mesh_batch_build(const mp_plan *const *plans, int32_t n, mp_plan **out)
{
    if (!out) return MP_EINVAL;
    *out = nullptr;
    if (!plans || n < 1) return MP_EINVAL;
    const mp_plan &P0 = *plans[0];
    for (int k = 0; k < n; ++k) {
        const mp_plan *P = plans[k];
        if (!P || P->opts.coloring != MP_COLOR_HIER || P->nmaps != P0.nmaps || P->ntosets != P0.ntosets ||
            P->lmap_stride != P0.lmap_stride || P->opts.layout != MP_LAYOUT_AOS)
            return MP_EINVAL;
        for (int m = 0; m < P0.nmaps; ++m)
            if (P->maps[m].arity != P0.maps[m].arity || P->maps[m].written != P0.maps[m].written ||
                P->maps[m].slot != P0.maps[m].slot || P->maps[m].to_set != P0.maps[m].to_set)
                return MP_EINVAL;
    }
    mp_plan *B = new (std::nothrow) mp_plan();
    if (!B) return MP_ENOMEM;
    try {
        B->opts = P0.opts;
        B->nmaps = P0.nmaps;
        B->ntosets = P0.ntosets;
        B->lmap_stride = P0.lmap_stride;
        int64_t from_total = 0, to_total[MP_MAX_TOSETS] = {0, 0};
        int32_t max_bs = 0, ncolors = 0;
        for (int k = 0; k < n; ++k) {
            from_total += plans[k]->from_size;
            for (int s = 0; s < B->ntosets; ++s) to_total[s] += plans[k]->toset_size[s];
            max_bs = std::max(max_bs, plans[k]->opts.block_size);
            ncolors = std::max(ncolors, plans[k]->ncolors);
        }
        if (from_total > INT32_MAX || to_total[0] > INT32_MAX || to_total[1] > INT32_MAX) throw std::bad_alloc();
        B->opts.block_size = max_bs;
        B->from_size = from_total;
        for (int s = 0; s < B->ntosets; ++s) {
            B->toset_id[s] = P0.toset_id[s];
            B->toset_size[s] = to_total[s];
        }
        for (int m = 0; m < B->nmaps; ++m) {
            B->maps[m] = mp_map_info{};
            B->maps[m].to_set = P0.maps[m].to_set;
            B->maps[m].arity = P0.maps[m].arity;
            B->maps[m].written = P0.maps[m].written;
            B->maps[m].slot = P0.maps[m].slot;
            B->maps[m].to_size = to_total[P0.maps[m].slot];
        }
        // per-mesh bases of every to-set in the concatenated data
        int64_t to_base[MP_MAX_TOSETS] = {0, 0};
        std::vector<int64_t> tob[MP_MAX_TOSETS], items_of(n);
        int64_t item_base = 0;
        for (int s = 0; s < MP_MAX_TOSETS; ++s) tob[s].resize(n);
        for (int k = 0; k < n; ++k) {
            items_of[k] = item_base;
            item_base += plans[k]->from_size;
            for (int s = 0; s < B->ntosets; ++s) {
                tob[s][k] = to_base[s];
                to_base[s] += plans[k]->toset_size[s];
                for (int32_t v : plans[k]->perm_to[s]) B->perm_to[s].push_back((int32_t)(v + tob[s][k]));
            }
        }
        // the device footprint array holds all meshes' slot-0 lists, then all
        // slot-1 lists; ids are offset into the concatenated data
        std::vector<int64_t> slot_base[MP_MAX_TOSETS];
        int64_t acc = 0;
        for (int s = 0; s < B->ntosets; ++s) {
            slot_base[s].resize(n);
            for (int k = 0; k < n; ++k) {
                slot_base[s][k] = acc;
                acc += (int64_t)plans[k]->fp_ids[s].size();
                for (int32_t v : plans[k]->fp_ids[s]) B->fp_ids[s].push_back((int32_t)(v + tob[s][k]));
            }
        }
        if (acc > INT32_MAX) throw std::bad_alloc();
        // gather rows follow the same concatenation, widened to the widest
        B->gat_w = 0;
        for (int k = 0; k < n; ++k) B->gat_w = std::max(B->gat_w, plans[k]->gat_w);
        for (int k = 0; k < n; ++k)
            if (plans[k]->gat_w == 0) B->gat_w = 0;
        if (B->gat_w > 0) {
            B->gat_tab.assign((size_t)acc * B->gat_w, 0xFFFF);
            for (int k = 0; k < n; ++k) {
                const mp_plan &P = *plans[k];
                int64_t own = 0;
                for (int s = 0; s < B->ntosets; ++s) {
                    const int64_t npt = (int64_t)P.fp_ids[s].size();
                    for (int64_t i = 0; i < npt; ++i)
                        for (int w = 0; w < P.gat_w; ++w)
                            B->gat_tab[(size_t)(slot_base[s][k] + i) * B->gat_w + w] =
                                P.gat_tab[(size_t)(own + i) * P.gat_w + w];
                    own += npt;
                }
            }
        }
        // blocks grouped by colour phase, meshes in order inside a phase; the
        // iterations of the union are renumbered to follow that block order,
        // so every block is a contiguous iteration range
        B->ncolors = ncolors;
        B->color_offsets.assign(1, 0);
        B->block_offsets.assign(1, 0);
        B->lmap.reserve((size_t)from_total * B->lmap_stride);
        B->thread_color.reserve(from_total);
        B->perm_from.reserve(from_total);
        int32_t next = 0;
        for (int c = 0; c < ncolors; ++c) {
            for (int k = 0; k < n; ++k) {
                const mp_plan &P = *plans[k];
                if (c >= P.ncolors) continue;
                for (int32_t b = P.color_offsets[c]; b < P.color_offsets[c + 1]; ++b) {
                    mp_block_desc d = P.desc[b];
                    const int32_t s0 = d.item_start;
                    for (int32_t it = s0; it < s0 + d.nitems; ++it) {
                        B->lmap.insert(B->lmap.end(), P.lmap.begin() + (size_t)it * P.lmap_stride,
                                       P.lmap.begin() + (size_t)(it + 1) * P.lmap_stride);
                        B->thread_color.push_back(P.thread_color[it]);
                        B->perm_from.push_back((int32_t)(P.perm_from[it] + items_of[k]));
                        for (int m = 0; m < B->nmaps; ++m) {
                            const mp_map_info &mi = P.maps[m];
                            for (int a = 0; a < mi.arity; ++a)
                                B->maps[m].idx.push_back((int32_t)(mi.idx[(int64_t)it * mi.arity + a] + tob[mi.slot][k]));
                        }
                    }
                    d.item_start = next;
                    next += d.nitems;
                    int64_t own_base = 0;  // the plan's fp_start indexes its own slot-major lists
                    for (int s = 0; s < B->ntosets; ++s) {
                        d.fp_start[s] = (int32_t)(d.fp_start[s] - own_base + slot_base[s][k]);
                        own_base += (int64_t)P.fp_ids[s].size();
                    }
                    B->desc.push_back(d);
                    B->block_color.push_back(c);
                    B->block_ncolors.push_back(P.block_ncolors[b]);
                    B->block_offsets.push_back(next);
                }
            }
            B->color_offsets.push_back((int32_t)B->desc.size());
        }
        if (next != from_total) throw std::bad_alloc();
        B->nblocks = (int32_t)B->desc.size();
        // statistics: maxima and sums over the meshes
        mp_plan_stats &S = B->stats;
        S = P0.stats;
        S.from_size = B->from_size;
        S.nblocks = B->nblocks;
        S.nblock_colors = B->ncolors;
        S.block_size = max_bs;
        S.max_thread_colors = 0;
        double tc = 0, acc_all = 0, uniq_all = 0, secs = 0;
        for (int s = 0; s < MP_MAX_TOSETS; ++s) {
            S.footprint_max[s] = 0;
            S.footprint_total[s] = 0;
            S.to_set_size[s] = s < B->ntosets ? B->toset_size[s] : 0;
        }
        double acc_s[MP_MAX_TOSETS] = {0, 0};
        for (int k = 0; k < n; ++k) {
            const mp_plan_stats &Q = plans[k]->stats;
            S.max_thread_colors = std::max(S.max_thread_colors, Q.max_thread_colors);
            tc += Q.mean_thread_colors * Q.nblocks;
            secs += Q.seconds_total;
            for (int s = 0; s < B->ntosets; ++s) {
                S.footprint_max[s] = std::max(S.footprint_max[s], Q.footprint_max[s]);
                S.footprint_total[s] += Q.footprint_total[s];
                acc_s[s] += Q.reuse[s] * Q.footprint_total[s];
                acc_all += Q.reuse[s] * Q.footprint_total[s];
                uniq_all += Q.footprint_total[s];
            }
        }
        for (int s = 0; s < B->ntosets; ++s)
            S.reuse[s] = S.footprint_total[s] ? acc_s[s] / S.footprint_total[s] : 0.0;
        S.reuse_all = uniq_all > 0 ? acc_all / uniq_all : 0.0;
        S.mean_thread_colors = B->nblocks ? tc / B->nblocks : 0.0;
        S.seconds_total = secs;
        S.plan_bytes = (int64_t)B->desc.size() * sizeof(mp_block_desc) + (int64_t)B->lmap.size() * 2 +
                       B->from_size + acc * 4;
    } catch (const std::bad_alloc &) {
        delete B;
        return MP_ENOMEM;
    }
    *out = B;
    return MP_OK;
}
