// Query planner (Sec. 6.1) and the schedule the executor runs.
//
// The planner builds the query graph (one vertex per variable and per
// distinct constant, one edge per triple pattern) and orders the edges in
// groups: the degree-driven traversal of Sec. 6.1.2 (with its constant
// variant) or the direction-driven traversal of Sec. 6.1.1 (with its cyclic
// variant). Where the text leaves a choice open the planner takes these
// readings: the root joins the visited set W when chosen; only vertices new
// to W are pushed; remaining ties go to the lower vertex (variables before
// constants, then by index), which wins a root choice and is pushed last so
// it is popped first; a popped vertex without unevaluated edges yields no
// group; with constants, when no unvisited vertex next to a constant is
// left, the root is chosen by the rule without constants.
//
// Schedule. One tree level per variable (Sec. 7.1, one path through all
// groups). Without a graph, variables are materialized in the order the
// groups reach them (a group's own vertex, then the new ends of its edges);
// with one, after the first level, by estimated candidates (greedy_levels). A variable's
// "binders" are its patterns to constants and to variables of earlier
// levels; each tree node takes its candidates from the shortest binder
// range and tests the others by membership. Its patterns to variables of
// later levels become pre-pruning tests (Sec. 7.2.2): presence of the
// predicate in the candidate's row / column, or the candidate vector of
// the triple scan (Eq. 17 / Eq. 21) when one was computed. A variable with
// a single pattern to another variable is not materialized (a leaf).
#include <algorithm>
#include <cstring>
#include <functional>
#include <set>

#include "gs_internal.h"

namespace gs {

namespace {

struct QVert {
    bool is_const;
    int64_t id;   // variable index or constant vertex id
    bool operator<(const QVert& o) const {
        if (is_const != o.is_const) return !is_const;   // variables first
        return id < o.id;
    }
    bool operator==(const QVert& o) const { return is_const == o.is_const && id == o.id; }
    int64_t code() const { return is_const ? -(1 + id) : id; }
};

struct QGraph {
    std::vector<QVert> V;                       // sorted
    std::vector<std::pair<int, int>> E;         // (subject vertex, object vertex) indices into V
};

int vindex(const QGraph& G, const QVert& v) {
    return (int)(std::lower_bound(G.V.begin(), G.V.end(), v) - G.V.begin());
}

QGraph make_graph(const int64_t* pat, uint32_t n) {
    QGraph G;
    std::set<QVert> vs;
    auto vk = [](int64_t x) { return x < 0 ? QVert{false, -x - 1} : QVert{true, x}; };
    for (uint32_t i = 0; i < n; ++i) { vs.insert(vk(pat[3 * i])); vs.insert(vk(pat[3 * i + 2])); }
    G.V.assign(vs.begin(), vs.end());
    for (uint32_t i = 0; i < n; ++i)
        G.E.push_back({vindex(G, vk(pat[3 * i])), vindex(G, vk(pat[3 * i + 2]))});
    return G;
}

struct Trav {
    const QGraph& G;
    std::vector<char> F;   // evaluated edges
    explicit Trav(const QGraph& g) : G(g), F(g.E.size(), 0) {}
    int n_out(int v) const { int c = 0; for (size_t i = 0; i < G.E.size(); ++i) c += !F[i] && G.E[i].first == v; return c; }
    int n_in(int v) const { int c = 0; for (size_t i = 0; i < G.E.size(); ++i) c += !F[i] && G.E[i].second == v; return c; }
    int n_inc(int v) const { int c = 0; for (size_t i = 0; i < G.E.size(); ++i) c += !F[i] && (G.E[i].first == v || G.E[i].second == v); return c; }
    bool all_done() const { for (char f : F) if (!f) return false; return true; }
};

using Groups = std::vector<std::pair<int, std::vector<int>>>;

// Sec. 6.1.2
void degree_driven(const QGraph& G, Groups& groups, std::vector<int>& roots) {
    Trav T(G);
    const int nv = (int)G.V.size();
    std::vector<char> W(nv, 0);
    bool has_const = false;
    for (int v = 0; v < nv; ++v) if (G.V[v].is_const) { W[v] = 1; has_const = true; }
    if (has_const) {   // constant variant of step 1: evaluate all edges of the constants
        for (int c = 0; c < nv; ++c) {
            if (!G.V[c].is_const) continue;
            std::vector<int> es;
            for (size_t i = 0; i < G.E.size(); ++i)
                if (!T.F[i] && (G.E[i].first == c || G.E[i].second == c)) es.push_back((int)i);
            if (es.empty()) continue;
            for (int i : es) T.F[i] = 1;
            groups.push_back({c, es});
        }
    }
    while (!T.all_done()) {
        std::vector<int> cand;
        for (int v = 0; v < nv; ++v) if (!W[v]) cand.push_back(v);
        if (has_const) {   // constant variant of step 2: next to a constant
            std::vector<int> adj;
            for (int v : cand) {
                bool a = false;
                for (auto& e : G.E)
                    if ((e.first == v && G.V[e.second].is_const) || (e.second == v && G.V[e.first].is_const)) a = true;
                if (a) adj.push_back(v);
            }
            if (!adj.empty()) cand = adj;
        }
        int root = -1, bi = -1, bo = -1;
        for (int v : cand) {   // cand is ascending, so strict '>' keeps the lower vertex on ties
            int ni = T.n_inc(v), no = T.n_out(v);
            if (root < 0 || ni > bi || (ni == bi && no > bo)) { root = v; bi = ni; bo = no; }
        }
        roots.push_back(root);
        W[root] = 1;
        std::vector<int> S{root};
        while (!S.empty()) {
            int v = S.back();
            S.pop_back();
            std::vector<int> es;
            for (size_t i = 0; i < G.E.size(); ++i)
                if (!T.F[i] && (G.E[i].first == v || G.E[i].second == v)) es.push_back((int)i);
            if (es.empty()) continue;
            for (int i : es) T.F[i] = 1;
            groups.push_back({v, es});
            std::vector<int> nw;
            for (int i : es) {
                int w = G.E[i].first == v ? G.E[i].second : G.E[i].first;
                if (!W[w] && std::find(nw.begin(), nw.end(), w) == nw.end()) nw.push_back(w);
            }
            for (int w : nw) W[w] = 1;
            // ascending by (unevaluated edges, unevaluated out-edges), lower vertex last
            std::stable_sort(nw.begin(), nw.end(), [&](int a, int b) {
                int ia = T.n_inc(a), ib = T.n_inc(b);
                if (ia != ib) return ia < ib;
                int oa = T.n_out(a), ob = T.n_out(b);
                if (oa != ob) return oa < ob;
                return a > b;
            });
            for (int w : nw) S.push_back(w);
        }
    }
}

// Sec. 6.1.1
void direction_driven(const QGraph& G, Groups& groups, std::vector<int>& roots) {
    Trav T(G);
    const int nv = (int)G.V.size();
    std::vector<char> W(nv, 0);
    while (!T.all_done()) {
        int root = -1, bo = -1;
        for (int pass = 0; pass < 2 && root < 0; ++pass) {   // pass 1: cyclic variant
            for (int v = 0; v < nv; ++v) {
                if (W[v]) continue;
                if (pass == 0 && T.n_in(v) > 0) continue;
                int no = T.n_out(v);
                if (root < 0 || no > bo) { root = v; bo = no; }
            }
        }
        roots.push_back(root);
        W[root] = 1;
        std::vector<int> S{root};
        while (!S.empty()) {
            int v = S.back();
            S.pop_back();
            std::vector<int> es;
            for (size_t i = 0; i < G.E.size(); ++i)
                if (!T.F[i] && G.E[i].first == v) es.push_back((int)i);
            if (es.empty()) continue;
            for (int i : es) T.F[i] = 1;
            groups.push_back({v, es});
            std::vector<int> nw;
            for (int i : es) {
                int w = G.E[i].second;
                if (!W[w] && std::find(nw.begin(), nw.end(), w) == nw.end()) nw.push_back(w);
            }
            for (int w : nw) W[w] = 1;
            std::stable_sort(nw.begin(), nw.end(), [&](int a, int b) {
                int oa = T.n_out(a), ob = T.n_out(b);
                if (oa != ob) return oa < ob;
                return a > b;
            });
            for (int w : nw) S.push_back(w);
        }
    }
}

}  // namespace

// Binding-tree paths of Sec. 7.1 (Ex. 7.1): from each root, follow each
// edge of its group to the other end; continue into that end's group when
// this edge is the one that first reached it, else the path ends there.
// Self-loops are checks at their variable's level and edges to constants
// are its binders, so neither is a path step: a path also ends at a
// variable whose group holds nothing else. A variable's group that no walk
// enters (a constant's edge reached it first) starts paths of its own.
static void make_paths(const QGraph& G, const Groups& groups, const std::vector<int>& roots, gs_plan* P) {
    std::vector<int> group_of(G.V.size(), -1);
    for (size_t i = 0; i < groups.size(); ++i) group_of[groups[i].first] = (int)i;
    std::vector<int> reached_by(G.V.size(), -1);
    std::vector<char> is_root(G.V.size(), 0);
    for (int r : roots) is_root[r] = 1;
    for (auto& gr : groups)
        for (int e : gr.second) {
            const int a = G.E[e].first, b = G.E[e].second;
            const int w = a == gr.first ? b : a;
            if (w == gr.first || G.V[w].is_const || is_root[w] || reached_by[w] >= 0) continue;
            reached_by[w] = e;
        }
    std::vector<int> vars, pats;
    std::vector<char> entered(G.V.size(), 0);
    // returns whether a path was recorded below v
    std::function<bool(int)> walk = [&](int v) {
        bool any = false;
        if (group_of[v] < 0) return any;
        entered[v] = 1;
        for (int e : groups[group_of[v]].second) {
            const int a = G.E[e].first, b = G.E[e].second;
            const int w = a == v ? b : a;
            if (w == v || G.V[w].is_const) continue;
            vars.push_back((int)G.V[w].id);
            pats.push_back(e);
            // into w's group when this edge first reached w; the path ends
            // at w when nothing follows there (only self-loops or constants)
            if (!(group_of[w] >= 0 && reached_by[w] == e && walk(w))) {
                P->paths.push_back(vars);
                P->path_pat.push_back(pats);
            }
            any = true;
            vars.pop_back();
            pats.pop_back();
        }
        return any;
    };
    for (int r : roots) {
        if (G.V[r].is_const) continue;
        vars.assign(1, (int)G.V[r].id);
        pats.assign(1, -1);
        walk(r);
    }
    // the group of a variable that a constant's edge reached first is
    // entered by no walk: its paths start at that variable
    for (auto& gr : groups) {
        if (G.V[gr.first].is_const || entered[gr.first]) continue;
        vars.assign(1, (int)G.V[gr.first].id);
        pats.assign(1, -1);
        walk(gr.first);
    }
    std::vector<char> covered(P->n_vars, 0);
    for (auto& pth : P->paths)
        for (int v : pth) covered[v] = 1;
    for (int v = 0; v < P->n_vars; ++v)
        if (!covered[v]) { P->paths.push_back({v}); P->path_pat.push_back({-1}); }
}

// Level order by estimated candidates. The first level stays the
// traversal's (the root, or the variable its first constant binds); then,
// repeatedly, the variable whose cheapest edge to a bound end (an earlier
// level or a constant) has the shortest mean range, from the graph's label
// statistics: a variable reachable only through frequent predicates waits
// until a rarer edge binds it, which keeps the binding tree small (its
// frequent edge becomes a membership test). Ties keep the traversal order;
// a variable with no edge to a bound end (another component) comes when
// nothing else is left. The answers do not depend on the order.
void greedy_levels(const gs_graph* g, const int64_t* pat, uint32_t n, std::vector<int>* order) {
    const std::vector<int> trav = *order;
    const double M = std::max<double>(1.0, (double)g->M);
    auto stat = [&](const std::vector<uint64_t>& v, uint32_t p) { return p < v.size() ? (double)v[p] : 0.0; };
    // mean range of label p in the row (dir 0) or column (dir 1) of a bound end
    auto fanout = [&](uint32_t p, int dir) {
        const double r = stat(g->lab_rows[dir], p);
        return r > 0 ? stat(g->lab_cnt[dir], p) / r : 0.0;
    };
    auto from_const = [&](uint32_t c, uint32_t p, int dir) {
        const std::vector<uint32_t>& deg = dir == 0 ? g->deg_out : g->deg_in;
        return c < deg.size() ? deg[c] * stat(g->lab_cnt[dir], p) / M : 0.0;
    };
    auto var_of = [](int64_t x) { return x < 0 ? (int)(-x - 1) : -1; };
    int k = 0;
    for (int v : trav) k = std::max(k, v + 1);
    std::vector<char> done(k, 0);
    std::vector<int> out{trav[0]};
    done[trav[0]] = 1;
    while (out.size() < trav.size()) {
        int best = -1;
        double best_f = 0.0;
        for (int v : trav) {
            if (done[v]) continue;
            double f = 1e300;
            for (uint32_t i = 0; i < n; ++i) {
                const int a = var_of(pat[3 * i]), b = var_of(pat[3 * i + 2]);
                const uint32_t p = (uint32_t)pat[3 * i + 1];
                if (a == v && b != v) {   // v the subject: candidates in the object's column
                    if (b < 0) f = std::min(f, from_const((uint32_t)pat[3 * i + 2], p, 1));
                    else if (done[b]) f = std::min(f, fanout(p, 1));
                }
                if (b == v && a != v) {   // v the object: candidates in the subject's row
                    if (a < 0) f = std::min(f, from_const((uint32_t)pat[3 * i], p, 0));
                    else if (done[a]) f = std::min(f, fanout(p, 0));
                }
            }
            if (f >= 1e300) continue;
            if (best < 0 || f < best_f) { best = v; best_f = f; }
        }
        if (best < 0)
            for (int v : trav)
                if (!done[v]) { best = v; break; }
        out.push_back(best);
        done[best] = 1;
    }
    *order = out;
}

gs_status make_plan(const gs_graph* g, const int64_t* pat, uint32_t n, uint32_t flags,
                    gs_plan** out) {
    *out = nullptr;
    if (!pat || n == 0 || n > (uint32_t)kMaxPatterns) {
        set_error("gs_plan_query: need 1..%d patterns", kMaxPatterns);
        return GS_EINVAL;
    }
    if ((flags & ~(GS_PLAN_DIRECTION | GS_PLAN_LISTS | GS_PLAN_PATHS)) != 0) { set_error("gs_plan_query: unknown flags %u", flags); return GS_EINVAL; }
    const uint32_t N = g ? g->N : 0xffffffffu, NP = g ? g->P : 65535u;
    int k = 0;
    std::vector<char> used(kMaxVars + 1, 0);
    for (uint32_t i = 0; i < n; ++i) {
        int64_t p = pat[3 * i + 1];
        if (p < 1 || p > (int64_t)NP) { set_error("gs_plan_query: pattern %u predicate %lld outside 1..%u", i, (long long)p, NP); return GS_EINVAL; }
        for (int j : {0, 2}) {
            int64_t x = pat[3 * i + j];
            if (x >= 0) {
                if (x >= (int64_t)N || x >= (1ll << 31)) { set_error("gs_plan_query: pattern %u vertex %lld out of range", i, (long long)x); return GS_EINVAL; }
            } else {
                int64_t v = -x - 1;
                if (v >= kMaxVars) { set_error("gs_plan_query: at most %d variables", kMaxVars); return GS_EINVAL; }
                used[v] = 1;
                k = std::max<int>(k, (int)v + 1);
            }
        }
    }
    if (k == 0) { set_error("gs_plan_query: the query has no variable"); return GS_EINVAL; }
    for (int v = 0; v < k; ++v)
        if (!used[v]) { set_error("gs_plan_query: variables must be numbered 0..K-1 (variable %d unused)", v); return GS_EINVAL; }

    gs_plan* P = new gs_plan();
    P->N = g ? g->N : 0; P->P = g ? g->P : 0; P->flags = flags; P->n_vars = k;
    P->patterns.assign(pat, pat + 3 * (size_t)n);

    QGraph G = make_graph(pat, n);
    Groups groups;
    std::vector<int> roots;
    bool has_const = false;
    for (auto& v : G.V) has_const |= v.is_const;
    if ((flags & GS_PLAN_DIRECTION) && !has_const) direction_driven(G, groups, roots);
    else degree_driven(G, groups, roots);
    for (auto& gr : groups) P->groups.push_back({G.V[gr.first].code(), gr.second});
    for (int r : roots) P->roots.push_back(G.V[r].code());
    make_paths(G, groups, roots, P);

    // ---- schedule ----
    auto var_of = [&](int64_t x) { return x < 0 ? (int)(-x - 1) : -1; };
    std::vector<int> deg(k, 0);
    std::vector<char> is_root(k, 0);
    for (int r : roots) if (!G.V[r].is_const) is_root[G.V[r].id] = 1;
    for (uint32_t i = 0; i < n; ++i) {
        int a = var_of(pat[3 * i]), b = var_of(pat[3 * i + 2]);
        if (a >= 0) deg[a]++;
        if (b >= 0 && b != a) deg[b]++;
        if (a >= 0 && a == b) deg[a]++;   // a self-loop is never a leaf edge
    }
    std::vector<int> leaf_pat(k, -1);
    for (int v = 0; v < k; ++v) {
        if (deg[v] != 1 || is_root[v]) continue;
        for (uint32_t i = 0; i < n; ++i) {
            int a = var_of(pat[3 * i]), b = var_of(pat[3 * i + 2]);
            if ((a == v && b >= 0 && b != v) || (b == v && a >= 0 && a != v)) leaf_pat[v] = (int)i;
        }
    }
    // two leaves joined by one pattern cannot both stay leaves
    for (int v = 0; v < k; ++v) {
        if (leaf_pat[v] < 0) continue;
        int i = leaf_pat[v];
        int a = var_of(pat[3 * i]), b = var_of(pat[3 * i + 2]);
        int w = a == v ? b : a;
        if (leaf_pat[w] >= 0) leaf_pat[std::max(v, w)] = -1;
    }
    std::vector<int> level_of(k, -1), order;
    auto materialize = [&](int v) {
        if (v < 0 || level_of[v] >= 0 || leaf_pat[v] >= 0) return;
        level_of[v] = (int)order.size();
        order.push_back(v);
    };
    for (auto& gr : groups) {
        const QVert& gv = G.V[gr.first];
        if (!gv.is_const) materialize((int)gv.id);
        for (int e : gr.second) {
            int a = G.E[e].first, b = G.E[e].second;
            int w = a == gr.first ? b : a;
            if (!G.V[w].is_const) materialize((int)G.V[w].id);
        }
    }
    for (int v = 0; v < k; ++v) materialize(v);   // not reached by any group (cannot happen)
    if (g && !g->lab_rows[0].empty() && order.size() > 2) greedy_levels(g, pat, n, &order);
    for (size_t l = 0; l < order.size(); ++l) level_of[order[l]] = (int)l;
    P->n_levels = (int)order.size();
    bool need_scan = false, too_many_probes = false;
    for (int l = 0; l < P->n_levels; ++l) {
        LevelSpec& L = P->levels[l];
        std::memset(&L, 0, sizeof(L));
        int w = order[l];
        L.var = w;
        L.vec = l;
        for (uint32_t i = 0; i < n; ++i) {
            int64_t s = pat[3 * i], o = pat[3 * i + 2];
            uint32_t p = (uint32_t)pat[3 * i + 1];
            int a = var_of(s), b = var_of(o);
            if (a == w && b == w) {
                bool dup = false;   // a repeated pattern adds no constraint
                for (int j = 0; j < L.n_self; ++j) dup |= L.self_label[j] == p;
                if (dup) continue;
                if (L.n_self >= kMaxSelf) { delete P; set_error("gs_plan_query: more than %d self-loop patterns on one variable", kMaxSelf); return GS_ENOTIMPL; }
                L.self_label[L.n_self++] = p;
                continue;
            }
            if (a != w && b != w) continue;
            bool w_is_subject = a == w;
            int other = w_is_subject ? b : a;
            int64_t other_const = w_is_subject ? o : s;
            bool bound = other < 0 || (level_of[other] >= 0 && level_of[other] < l);
            if (bound) {
                bool dup = false;
                for (int j = 0; j < L.n_binders; ++j) {
                    const Binder& B = L.b[j];
                    dup |= B.label == p && B.dir == (w_is_subject ? 1 : 0) &&
                           (other < 0 ? (B.from_const && B.c == (uint32_t)other_const)
                                      : (!B.from_const && B.level == level_of[other]));
                }
                if (dup) continue;
                if (L.n_binders >= kMaxBinders) { delete P; set_error("gs_plan_query: more than %d edges join one variable to bound ends", kMaxBinders); return GS_ENOTIMPL; }
                Binder& B = L.b[L.n_binders++];
                B.label = p;
                B.from_const = other < 0;
                B.c = other < 0 ? (uint32_t)other_const : 0;
                B.level = other < 0 ? -1 : (int16_t)level_of[other];
                B.dir = w_is_subject ? 1 : 0;
            } else {
                bool dup = false;
                for (int j = 0; j < L.n_probes; ++j)
                    dup |= L.pr[j].label == p && L.pr[j].dir == (w_is_subject ? 0u : 1u);
                if (dup) continue;
                if (L.n_probes >= kMaxProbes) { too_many_probes = true; continue; }
                L.pr[L.n_probes].label = p;
                L.pr[L.n_probes].dir = w_is_subject ? 0 : 1;
                L.n_probes++;
            }
        }
        L.src = L.n_binders > 0 ? kSrcBinders : kSrcList;
        if (L.src == kSrcList) need_scan = true;
    }
    if (too_many_probes) need_scan = true;
    for (int v = 0; v < k; ++v) P->var_src[v] = level_of[v];
    P->n_leaves = 0;
    for (int v = 0; v < k; ++v) {
        if (leaf_pat[v] < 0) continue;
        int i = leaf_pat[v];
        int a = var_of(pat[3 * i]), b = var_of(pat[3 * i + 2]);
        LeafSpec& F = P->leaves[P->n_leaves];
        F.var = v;
        F.label = (uint32_t)pat[3 * i + 1];
        int anchor = a == v ? b : a;
        F.level = level_of[anchor];
        F.dir = (b == v) ? 0 : 1;     // leaf is the object -> CSR row of the anchor
        P->var_src[v] = -(P->n_leaves + 1);
        P->n_leaves++;
    }
    for (uint32_t i = 0; i < n; ++i)
        if (pat[3 * i] >= 0 && pat[3 * i + 2] >= 0) {
            P->const_triples.push_back((uint32_t)pat[3 * i]);
            P->const_triples.push_back((uint32_t)pat[3 * i + 1]);
            P->const_triples.push_back((uint32_t)pat[3 * i + 2]);
        }

    P->needs_scan = need_scan;
    if (need_scan) {
        // Bitmap form: candidate vectors of every materialized variable over
        // all its patterns. List form: vectors only for the levels listed
        // from one (roots); the other levels keep their probes.
        auto slot = [&](uint32_t* preds, int32_t& cnt, uint32_t p) -> int {
            for (int j = 0; j < cnt; ++j) if (preds[j] == p) return j;
            if (cnt >= kMaxSlots) return -1;
            preds[cnt] = p;
            return cnt++;
        };
        auto make_scan = [&](ScanSpec& S, bool roots_only) -> gs_status {
            std::memset(&S, 0, sizeof(S));
            for (int l = 0; l < P->n_levels; ++l) {
                if (roots_only && P->levels[l].src != kSrcList) continue;
                int w = order[l];
                int bi = S.n_bvars++;
                S.bvar[bi] = w;
                S.blevel[bi] = l;
                for (uint32_t i = 0; i < n; ++i) {
                    int a = var_of(pat[3 * i]), b = var_of(pat[3 * i + 2]);
                    uint32_t p = (uint32_t)pat[3 * i + 1];
                    if (a == w) {
                        int s = slot(S.out_pred, S.n_out, p);
                        if (s < 0) { set_error("gs_plan_query: more than %d distinct out-predicates", kMaxSlots); return GS_ENOTIMPL; }
                        S.need_out[bi] |= 1u << s;
                    }
                    if (b == w) {
                        int s = slot(S.in_pred, S.n_in, p);
                        if (s < 0) { set_error("gs_plan_query: more than %d distinct in-predicates", kMaxSlots); return GS_ENOTIMPL; }
                        S.need_in[bi] |= 1u << s;
                    }
                }
            }
            return GS_OK;
        };
        gs_status rc = make_scan(P->scan, false);
        if (rc == GS_OK && !too_many_probes) rc = make_scan(P->scan_alt, true);
        if (rc != GS_OK) { delete P; return rc; }
        P->list_ok = !too_many_probes;
        for (int l = 0; l < P->n_levels; ++l) {
            P->levels_alt[l] = P->levels[l];          // list form: the probes stay
            P->levels[l].use_bitmap = 1;
            P->levels[l].n_probes = 0;
        }
        if ((flags & GS_PLAN_LISTS) && P->list_ok) switch_frontier_form(P);
    }
    if (flags & GS_PLAN_PATHS) {
        // per-path trees test every step against its variable's candidate
        // vector: one vector per variable (vector v for variable v)
        ScanSpec& S = P->path_scan;
        std::memset(&S, 0, sizeof(S));
        auto slot = [&](uint32_t* preds, int32_t& cnt, uint32_t p) -> int {
            for (int j = 0; j < cnt; ++j) if (preds[j] == p) return j;
            if (cnt >= kMaxSlots) return -1;
            preds[cnt] = p;
            return cnt++;
        };
        for (int v = 0; v < k; ++v) {
            S.bvar[v] = v;
            S.blevel[v] = v;
            S.n_bvars = v + 1;
            for (uint32_t i = 0; i < n; ++i) {
                const int a = var_of(pat[3 * i]), b = var_of(pat[3 * i + 2]);
                const uint32_t p = (uint32_t)pat[3 * i + 1];
                int sl = 0;
                if (a == v && (sl = slot(S.out_pred, S.n_out, p)) >= 0) S.need_out[v] |= 1u << sl;
                if (a == v && sl < 0) { delete P; set_error("gs_plan_query: more than %d distinct out-predicates", kMaxSlots); return GS_ENOTIMPL; }
                if (b == v && (sl = slot(S.in_pred, S.n_in, p)) >= 0) S.need_in[v] |= 1u << sl;
                if (b == v && sl < 0) { delete P; set_error("gs_plan_query: more than %d distinct in-predicates", kMaxSlots); return GS_ENOTIMPL; }
            }
        }
    }
    *out = P;
    return GS_OK;
}

bool switch_frontier_form(gs_plan* P) {
    if (!P->needs_scan || !P->list_ok) return false;
    for (int l = 0; l < P->n_levels; ++l) std::swap(P->levels[l], P->levels_alt[l]);
    std::swap(P->scan, P->scan_alt);
    P->list_form = !P->list_form;
    return true;
}

}  // namespace gs
