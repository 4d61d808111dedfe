// Database sharding over several GPUs: the partition and the one exchange
// step (host code only; no kernel here).
//
// The paper leaves multi-GPU execution to future work (Section 5); SW#db
// itself spreads a search over GPU(s) (Section 2.3).  Every (query,
// database sequence) score is independent of every other, so the database
// splits into shards that separate GPUs search with the full query batch,
// each keeping its own top-k.  The only exchange is then per query: gather
// the shards' k best (score, index) and merge them.  This file holds the
// two host steps of that flow:
//
// * sw_shard_plan: a partition of the database that balances residues (the
//   work of a shard is its residue count times the query residues) and
//   spreads every length range over all shards, so that each shard's
//   length-sorted layout looks like the whole database's.  Sequences are
//   dealt longest first, each to the shard holding the fewest residues so
//   far (ties to the lower shard number); a shard lists its members in the
//   caller's order, so ordering by a shard's local index is ordering by
//   the caller's index.
// * sw_hits_merge: the global top-k of each query from the shards' top-k
//   lists.  It is exact: a sequence outside its own shard's k best has k
//   better sequences in that shard alone, so it cannot be among the k best
//   overall; and within a shard the local order is the caller's order, so
//   the tie order (score descending, then caller's index ascending) of the
//   merged list is the tie order of an unsharded search.
#include <algorithm>
#include <cstring>
#include <functional>
#include <queue>
#include <vector>

#include "../../include/swdb.h"
#include "swdb_internal.cuh"

extern "C" int sw_shard_plan(const int64_t *offsets, int64_t n_seqs, int32_t n_shards, int64_t *members,
                             int64_t *member_offsets) {
    using swdb::set_error;
    set_error(SW_OK, "");
    if (!offsets || !member_offsets || (n_seqs > 0 && !members)) return set_error(SW_ERR_INVALID_ARG, "NULL argument");
    if (n_seqs < 0) return set_error(SW_ERR_INVALID_ARG, "n_seqs < 0");
    if (n_shards < 1) return set_error(SW_ERR_INVALID_ARG, "n_shards must be >= 1");
    for (int64_t i = 0; i < n_seqs; ++i)
        if (offsets[i + 1] < offsets[i]) return set_error(SW_ERR_INVALID_ARG, "offsets must be non-decreasing");
    std::vector<int64_t> order(static_cast<size_t>(n_seqs));
    for (int64_t i = 0; i < n_seqs; ++i) order[size_t(i)] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
        return offsets[x + 1] - offsets[x] > offsets[y + 1] - offsets[y];
    });
    // (residues so far, shard): the smallest pair first
    using Load = std::pair<int64_t, int32_t>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int32_t s = 0; s < n_shards; ++s) heap.push({0, s});
    std::vector<int32_t> shard_of(static_cast<size_t>(n_seqs));
    std::vector<int64_t> count(size_t(n_shards), 0);
    for (int64_t t : order) {
        Load l = heap.top();
        heap.pop();
        shard_of[size_t(t)] = l.second;
        ++count[size_t(l.second)];
        l.first += offsets[t + 1] - offsets[t];
        heap.push(l);
    }
    member_offsets[0] = 0;
    for (int32_t s = 0; s < n_shards; ++s) member_offsets[s + 1] = member_offsets[s] + count[size_t(s)];
    std::vector<int64_t> fill(member_offsets, member_offsets + n_shards);
    for (int64_t i = 0; i < n_seqs; ++i) members[fill[size_t(shard_of[size_t(i)])]++] = i;   // caller's order
    return SW_OK;
}

extern "C" int sw_hits_merge(const sw_hit *shard_hits, const int64_t *members, const int64_t *member_offsets,
                             int32_t n_shards, int32_t n_q, int32_t top_k, sw_hit *hits_out) {
    using swdb::set_error;
    set_error(SW_OK, "");
    if (n_shards < 1 || n_q < 0 || top_k < 0) return set_error(SW_ERR_INVALID_ARG, "bad count");
    if (n_q == 0 || top_k == 0) return SW_OK;
    if (!shard_hits || !member_offsets || !hits_out) return set_error(SW_ERR_INVALID_ARG, "NULL argument");
    if (member_offsets[0] != 0) return set_error(SW_ERR_INVALID_ARG, "member_offsets[0] must be 0");
    for (int32_t s = 0; s < n_shards; ++s)
        if (member_offsets[s + 1] < member_offsets[s]) return set_error(SW_ERR_INVALID_ARG, "member_offsets must be non-decreasing");
    if (member_offsets[n_shards] > 0 && !members) return set_error(SW_ERR_INVALID_ARG, "members is NULL");
    const size_t per_shard = size_t(n_q) * size_t(top_k);
    // validate every shard-local index first, so that no output is written on error
    for (int32_t s = 0; s < n_shards; ++s) {
        const int64_t n_s = member_offsets[s + 1] - member_offsets[s];
        const sw_hit *h = shard_hits + size_t(s) * per_shard;
        for (size_t i = 0; i < per_shard; ++i)
            if (h[i].db_index < -1 || h[i].db_index >= n_s)
                return set_error(SW_ERR_INVALID_ARG, "a shard hit's db_index is outside its shard");
    }
    std::vector<int32_t> head(static_cast<size_t>(n_shards));
    for (int32_t q = 0; q < n_q; ++q) {
        std::fill(head.begin(), head.end(), 0);
        for (int32_t r = 0; r < top_k; ++r) {
            int32_t best = -1;
            int32_t best_score = 0;
            int64_t best_index = 0;
            for (int32_t s = 0; s < n_shards; ++s) {
                if (head[size_t(s)] >= top_k) continue;
                const sw_hit &h = shard_hits[size_t(s) * per_shard + size_t(q) * top_k + size_t(head[size_t(s)])];
                if (h.db_index < 0) continue;                      // the shard has no more hits
                const int64_t g = members[member_offsets[s] + h.db_index];
                if (best < 0 || h.score > best_score || (h.score == best_score && g < best_index)) {
                    best = s;
                    best_score = h.score;
                    best_index = g;
                }
            }
            sw_hit &o = hits_out[size_t(q) * top_k + size_t(r)];
            o.reserved = 0;
            if (best < 0) {
                o.score = -1;
                o.db_index = -1;
            } else {
                o.score = best_score;
                o.db_index = best_index;
                ++head[size_t(best)];
            }
        }
    }
    return SW_OK;
}

extern "C" int sw_scores_scatter(const int32_t *shard_scores, const int64_t *members, int64_t n_members, int32_t n_q,
                                 int64_t n_seqs, int32_t *scores_out) {
    using swdb::set_error;
    set_error(SW_OK, "");
    if (n_q < 0 || n_members < 0 || n_seqs < 0) return set_error(SW_ERR_INVALID_ARG, "bad count");
    if (n_q == 0 || n_members == 0) return SW_OK;
    if (!shard_scores || !members || !scores_out) return set_error(SW_ERR_INVALID_ARG, "NULL argument");
    for (int64_t j = 0; j < n_members; ++j)
        if (members[j] < 0 || members[j] >= n_seqs) return set_error(SW_ERR_INVALID_ARG, "member index out of range");
    for (int32_t q = 0; q < n_q; ++q) {
        const int32_t *src = shard_scores + size_t(q) * size_t(n_members);
        int32_t *dst = scores_out + size_t(q) * size_t(n_seqs);
        for (int64_t j = 0; j < n_members; ++j) dst[members[j]] = src[j];
    }
    return SW_OK;
}
