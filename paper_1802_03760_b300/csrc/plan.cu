// Query plan compiler (host). Turns Q := E(a_s, a_d), ... and a global
// attribute order into, per extension level, the atoms that bind the new
// attribute and which index each one reads (Section 2.2: the relations
// containing a_{j+1}; Section 4.1: an atom E(a_k, a_{j+1}) with a_k bound
// reads the out-neighbours of x_k, an atom E(a_{j+1}, a_k) the
// in-neighbours). Evaluation starts from the edges of an atom over the
// first two attributes (Section 4.2).
#include "gj_internal.cuh"

int gj_plan_compile(const uint32_t* as, const uint32_t* ad, uint32_t natoms, uint32_t k, const uint32_t* order,
                    Plan* p, std::string* why) {
    auto bad = [&](const char* m) {
        if (why) *why = m;
        return GJ_E_INVALID;
    };
    if (k < 2 || k > GJ_MAX_K) return bad("k must be in [2, 8]");
    if (natoms < 1 || natoms > GJ_MAX_ATOMS) return bad("n_atoms must be in [1, 16]");
    memset(p, 0, sizeof(*p));
    p->k = k;
    p->natoms = natoms;
    uint32_t used = 0;
    for (uint32_t t = 0; t < natoms; t++) {
        if (as[t] >= k || ad[t] >= k) return bad("atom attribute out of range");
        if (as[t] == ad[t]) return bad("atom with equal attributes");
        used |= (1u << as[t]) | (1u << ad[t]);
    }
    if (used != (1u << k) - 1) return bad("an attribute appears in no atom");
    uint32_t seen = 0;
    for (uint32_t j = 0; j < k; j++) {
        uint32_t a = order ? order[j] : j;
        if (a >= k || (seen & (1u << a))) return bad("order is not a permutation of the attributes");
        seen |= 1u << a;
        p->order[j] = a;
        p->qpos[a] = j;
    }
    // seed atom and filters over the first two positions
    bool have_seed = false;
    for (uint32_t t = 0; t < natoms; t++) {
        uint32_t ps = p->qpos[as[t]], pd = p->qpos[ad[t]];
        if (ps > 1 || pd > 1) continue;
        uint32_t dir = (ps == 0) ? 0u : 1u;  // 0: E(x0, x1)
        if (!have_seed) {
            p->seed_atom = t;
            p->seed_dir = dir;
            have_seed = true;
        } else {
            p->sf_dir[p->nsf] = (uint8_t)dir;
            p->sf_atom[p->nsf] = (uint8_t)t;
            p->nsf++;
        }
    }
    if (!have_seed) return bad("the first two attributes of the order share no atom");
    for (uint32_t j = 2; j < k; j++) {
        uint32_t nb = 0;
        for (uint32_t t = 0; t < natoms; t++) {
            uint32_t ps = p->qpos[as[t]], pd = p->qpos[ad[t]];
            if (pd == j && ps < j) {  // E(x_ps, x_j): out-neighbours of x_ps
                p->bpos[j][nb] = (uint8_t)ps;
                p->bdir[j][nb] = 0;
                p->batom[j][nb] = (uint8_t)t;
                nb++;
            } else if (ps == j && pd < j) {  // E(x_j, x_pd): in-neighbours of x_pd
                p->bpos[j][nb] = (uint8_t)pd;
                p->bdir[j][nb] = 1;
                p->batom[j][nb] = (uint8_t)t;
                nb++;
            }
        }
        if (nb == 0) return bad("an attribute shares no atom with any earlier attribute of the order");
        p->nb[j] = nb;
    }
    return GJ_OK;
}

// Delta query dQ_i (Section 3.3.1): the attribute order starts with atom
// i's attributes (source, destination) and continues with, repeatedly, the
// first attribute in q's order that shares an atom with a bound one (the
// paper allows any order after R_i's attributes; this keeps every later
// level bound by at least one atom). Atoms before i in definition order read
// the new version, atoms after i the old one (Section 4.3); atom i itself
// is the seed, so its changes enter once, with their signs.
int gj_plan_compile_delta(const gj_query* q, uint32_t i, Plan* p, std::string* why) {
    auto bad = [&](const char* m) {
        if (why) *why = m;
        return GJ_E_INVALID;
    };
    const uint32_t k = q->k, natoms = q->natoms;
    if (i >= natoms) return bad("atom index out of range");
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
            p->sf_atom[p->nsf] = (uint8_t)t;
            p->sf_view[p->nsf] = (uint8_t)(t < i ? GJ_VIEW_NEW : GJ_VIEW_OLD);
            p->nsf++;
        }
    }
    for (uint32_t j = 2; j < k; j++) {
        uint32_t nb = 0;
        for (uint32_t t = 0; t < natoms; t++) {
            if (t == i) continue;
            uint32_t ps = p->qpos[q->as[t]], pd = p->qpos[q->ad[t]];
            int dir = -1;
            uint32_t bp = 0;
            if (pd == j && ps < j) { dir = 0; bp = ps; }
            else if (ps == j && pd < j) { dir = 1; bp = pd; }
            if (dir < 0) continue;
            p->bpos[j][nb] = (uint8_t)bp;
            p->bdir[j][nb] = (uint8_t)dir;
            p->batom[j][nb] = (uint8_t)t;
            p->bview[j][nb] = (uint8_t)(t < i ? GJ_VIEW_NEW : GJ_VIEW_OLD);
            nb++;
        }
        if (nb == 0) return bad("an attribute shares no atom with any earlier attribute of the order");
        p->nb[j] = nb;
    }
    return GJ_OK;
}
