// Query plan compiler (host). Turns Q := E(a_s, a_d), ..., tri(a_i, a_j,
// a_l), ... with inequalities x_a < x_b and a global attribute order into,
// per extension level, the relations that bind the new attribute and which
// index each one reads (Section 2.2: the relations containing a_{j+1};
// Section 4.1: an atom E(a_k, a_{j+1}) with a_k bound reads the
// out-neighbours of x_k, an atom E(a_{j+1}, a_k) the in-neighbours; Section
// 5.4: a tri atom reads the triangle list of its first two attributes and
// inequalities filter prefixes). Evaluation starts from the edges over the
// first two attributes (Section 4.2).
#include "gj_internal.cuh"

namespace {

// Inequality filters of level j (positions): every constraint between the
// attribute at position j and one at an earlier position.
bool add_filters(const gj_query* q, Plan* p, uint32_t j, std::string* why) {
    for (uint32_t t = 0; t < q->nlt; t++) {
        const uint32_t pa = p->qpos[q->la[t]], pb = p->qpos[q->lb[t]];
        uint32_t other, less;
        if (pa == j && pb < j) { other = pb; less = 1; }       // x_j < x_other
        else if (pb == j && pa < j) { other = pa; less = 0; }  // x_other < x_j
        else continue;
        if (p->nlt[j] >= GJ_MAX_LT) {
            if (why) *why = "more than 8 inequalities end at one attribute";
            return false;
        }
        p->lt_pos[j][p->nlt[j]] = (uint8_t)other;
        p->lt_less[j][p->nlt[j]] = (uint8_t)less;
        p->nlt[j]++;
    }
    return true;
}

// Bit p set for every position that the last level's lists and filters read.
uint32_t last_level_reads(const Plan* p) {
    const uint32_t j = p->k - 1;
    uint32_t m = 0;
    for (uint32_t b = 0; b < p->nb[j]; b++) {
        m |= 1u << p->bpos[j][b];
        if (p->bdir[j][b] == GJ_BIND_TRI) m |= 1u << p->bpos2[j][b];
    }
    for (uint32_t c = 0; c < p->nlt[j]; c++) m |= 1u << p->lt_pos[j][c];
    return m;
}

}  // namespace

bool gj_plan_ext(const Plan& p) {
    if (p.agg || p.fact) return true;
    for (uint32_t j = 1; j < p.k; j++) {
        if (p.nlt[j]) return true;
        for (uint32_t b = 0; j >= 2 && b < p.nb[j]; b++)
            if (p.bdir[j][b] == GJ_BIND_TRI) return true;
    }
    return false;
}

int gj_plan_compile(const gj_query* q, Plan* p, std::string* why) {
    auto bad = [&](const char* m) {
        if (why) *why = m;
        return GJ_E_INVALID;
    };
    const uint32_t k = q->k, natoms = q->natoms, ntri = q->ntri;
    if (k < 2 || k > GJ_MAX_K) return bad("k must be in [2, 8]");
    if (natoms + ntri < 1 || natoms > GJ_MAX_ATOMS || ntri > GJ_MAX_ATOMS || q->nlt > GJ_MAX_ATOMS)
        return bad("need 1..16 edge atoms or tri atoms and at most 16 inequalities");
    memset(p, 0, sizeof(*p));
    p->k = k;
    p->natoms = natoms;
    uint32_t used = 0;
    for (uint32_t t = 0; t < natoms; t++) {
        if (q->as[t] >= k || q->ad[t] >= k) return bad("atom attribute out of range");
        if (q->as[t] == q->ad[t]) return bad("atom with equal attributes");
        used |= (1u << q->as[t]) | (1u << q->ad[t]);
    }
    for (uint32_t t = 0; t < ntri; t++) {
        if (q->ta[t] >= k || q->tb[t] >= k || q->tc[t] >= k) return bad("tri atom attribute out of range");
        if (q->ta[t] == q->tb[t] || q->ta[t] == q->tc[t] || q->tb[t] == q->tc[t])
            return bad("tri atom with equal attributes");
        used |= (1u << q->ta[t]) | (1u << q->tb[t]) | (1u << q->tc[t]);
    }
    for (uint32_t t = 0; t < q->nlt; t++)
        if (q->la[t] >= k || q->lb[t] >= k || q->la[t] == q->lb[t]) return bad("inequality between equal or unknown attributes");
    if (used != (1u << k) - 1) return bad("an attribute appears in no atom");
    uint32_t seen = 0;
    for (uint32_t j = 0; j < k; j++) {
        uint32_t a = q->order[j];
        if (a >= k || (seen & (1u << a))) return bad("order is not a permutation of the attributes");
        seen |= 1u << a;
        p->order[j] = a;
        p->qpos[a] = j;
    }
    // seed: an edge atom over the first two positions, else a tri atom whose
    // first two attributes they are (its triangles lie on those edges);
    // further edge atoms over them filter the seeds
    bool have_seed = false;
    for (uint32_t t = 0; t < natoms; t++) {
        uint32_t ps = p->qpos[q->as[t]], pd = p->qpos[q->ad[t]];
        if (ps > 1 || pd > 1) continue;
        uint32_t dir = (ps == 0) ? 0u : 1u;  // 0: E(x0, x1)
        if (!have_seed) {
            p->seed_atom = t;
            p->seed_dir = dir;
            have_seed = true;
        } else {
            p->sf_dir[p->nsf] = (uint8_t)dir;
            p->nsf++;
        }
    }
    for (uint32_t t = 0; t < ntri && !have_seed; t++) {
        uint32_t pa = p->qpos[q->ta[t]], pb = p->qpos[q->tb[t]];
        if (pa > 1 || pb > 1) continue;
        p->seed_atom = GJ_MAX_ATOMS;  // no edge atom: the edges of the tri atom's first two attributes
        p->seed_dir = (pa == 0) ? 0u : 1u;
        have_seed = true;
    }
    if (!have_seed) return bad("the first two attributes of the order share no atom");
    for (uint32_t t = 0; t < ntri; t++)
        if (p->qpos[q->tc[t]] < p->qpos[q->ta[t]] || p->qpos[q->tc[t]] < p->qpos[q->tb[t]])
            return bad("a tri atom's third attribute must follow its first two in the order");
    if (!add_filters(q, p, 1, why)) return GJ_E_INVALID;
    for (uint32_t j = 2; j < k; j++) {
        uint32_t nb = 0;
        for (uint32_t t = 0; t < natoms; t++) {
            uint32_t ps = p->qpos[q->as[t]], pd = p->qpos[q->ad[t]];
            int dir = -1;
            uint32_t bp = 0;
            if (pd == j && ps < j) { dir = GJ_BIND_FWD; bp = ps; }       // E(x_ps, x_j): out-neighbours of x_ps
            else if (ps == j && pd < j) { dir = GJ_BIND_REV; bp = pd; }  // E(x_j, x_pd): in-neighbours of x_pd
            if (dir < 0) continue;
            if (nb >= GJ_MAX_BIND) return bad("more than 12 relations bind one attribute");
            p->bpos[j][nb] = (uint8_t)bp;
            p->bdir[j][nb] = (uint8_t)dir;
            nb++;
        }
        for (uint32_t t = 0; t < ntri; t++) {
            if (p->qpos[q->tc[t]] != j) continue;
            if (nb >= GJ_MAX_BIND) return bad("more than 12 relations bind one attribute");
            p->bpos[j][nb] = (uint8_t)p->qpos[q->ta[t]];
            p->bpos2[j][nb] = (uint8_t)p->qpos[q->tb[t]];
            p->bdir[j][nb] = GJ_BIND_TRI;
            nb++;
        }
        if (nb == 0) return bad("an attribute shares no atom with any earlier attribute of the order");
        p->nb[j] = nb;
        if (!add_filters(q, p, j, why)) return GJ_E_INVALID;
    }
    // Aggregation pays when the positions the last level does not read are
    // the most recently bound ones (a suffix k-1-s .. k-2 of the order): the
    // prefixes of a batch that share a parent then agree on everything the
    // last level reads and sit next to one another.
    if (k >= 3) {
        const uint32_t all = (1u << (k - 1)) - 1, reads = last_level_reads(p), skip = all & ~reads;
        const bool suffix = skip && ((skip + (skip & (0u - skip))) & all) == 0;  // one run of bits ending at k-2
        p->agg = suffix ? reads : 0u;
        // exactly position k-2 unread: its extensions factorise per parent
        // (subsumes the aggregation of equal neighbours at the last level)
        if (k >= 4 && skip == (1u << (k - 2))) {
            p->fact = 1;
            p->agg = 0;
        }
    }
    return GJ_OK;
}

// Delta query dQ_i (Section 3.3.1): the attribute order starts with atom
// i's attributes (source, destination) and continues with, repeatedly, the
// first attribute in q's order that shares an atom with a bound one (the
// paper allows any order after R_i's attributes; this keeps every later
// level bound by at least one atom). Atoms before i in definition order read
// the new version, atoms after i the old one (Section 4.3); atom i itself
// is the seed, so its changes enter once, with their signs. Inequalities
// filter as in the static plan. Queries with tri atoms have no delta plans.
int gj_plan_compile_delta(const gj_query* q, uint32_t i, Plan* p, std::string* why) {
    auto bad = [&](const char* m) {
        if (why) *why = m;
        return GJ_E_INVALID;
    };
    const uint32_t k = q->k, natoms = q->natoms;
    if (i >= natoms) return bad("atom index out of range");
    if (q->ntri) return bad("queries with tri atoms have no delta queries");
    memset(p, 0, sizeof(*p));
    p->k = k;
    p->natoms = natoms;
    p->delta = 1;
    uint32_t n = 0, bound = 0;
    auto bind = [&](uint32_t a) {
        p->order[n] = a;
        p->qpos[a] = n;
        n++;
        bound |= 1u << a;
    };
    bind(q->as[i]);
    bind(q->ad[i]);
    while (n < k) {
        bool found = false;
        for (uint32_t jj = 0; jj < k && !found; jj++) {
            uint32_t a = q->order[jj];
            if (bound & (1u << a)) continue;
            for (uint32_t t = 0; t < natoms; t++) {
                if ((q->as[t] == a && (bound & (1u << q->ad[t]))) || (q->ad[t] == a && (bound & (1u << q->as[t])))) {
                    found = true;
                    break;
                }
            }
            if (found) bind(a);
        }
        if (!found) return bad("the query graph is not connected");
    }
    p->seed_atom = i;
    p->seed_dir = 0;
    for (uint32_t t = 0; t < natoms; t++) {
        if (t == i) continue;
        uint32_t ps = p->qpos[q->as[t]], pd = p->qpos[q->ad[t]];
        if (ps <= 1 && pd <= 1) {
            p->sf_dir[p->nsf] = (uint8_t)(ps == 0 ? 0 : 1);
            p->sf_view[p->nsf] = (uint8_t)(t < i ? GJ_VIEW_NEW : GJ_VIEW_OLD);
            p->nsf++;
        }
    }
    if (!add_filters(q, p, 1, why)) return GJ_E_INVALID;
    for (uint32_t j = 2; j < k; j++) {
        uint32_t nb = 0;
        for (uint32_t t = 0; t < natoms; t++) {
            if (t == i) continue;
            uint32_t ps = p->qpos[q->as[t]], pd = p->qpos[q->ad[t]];
            int dir = -1;
            uint32_t bp = 0;
            if (pd == j && ps < j) { dir = GJ_BIND_FWD; bp = ps; }
            else if (ps == j && pd < j) { dir = GJ_BIND_REV; bp = pd; }
            if (dir < 0) continue;
            p->bpos[j][nb] = (uint8_t)bp;
            p->bdir[j][nb] = (uint8_t)dir;
            if (nb >= GJ_MAX_BIND) return bad("more than 12 relations bind one attribute");
            p->bview[j][nb] = (uint8_t)(t < i ? GJ_VIEW_NEW : GJ_VIEW_OLD);
            nb++;
        }
        if (nb == 0) return bad("an attribute shares no atom with any earlier attribute of the order");
        p->nb[j] = nb;
        if (!add_filters(q, p, j, why)) return GJ_E_INVALID;
    }
    return GJ_OK;
}
