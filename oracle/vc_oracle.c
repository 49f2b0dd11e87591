/*
 * Sequential CPU oracle for exact vertex cover by branch-and-reduce.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the GPU path is checked
 * against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * library never calls it, and it shares no code with the CUDA sources.
 *
 * What it computes (Yamout et al., "Parallel Vertex Cover Algorithms on GPUs"):
 *   - MVC: the size of a minimum vertex cover and one cover of that size (Sec. II-A).
 *   - PVC: whether a cover of size <= k exists, and one such cover when it does (Sec. II-A).
 * How: the recursive search of Sec. II-B (Fig. 1's algorithm, described in prose there):
 *   reduce to a fixpoint; stop check; if edgeless record the solution; else branch on the
 *   maximum-degree vertex v into "take v" and "take N(v)".  The incumbent starts at the greedy
 *   upper bound (Sec. II-B).  PVC uses k in place of best (Sec. II-B, last paragraph).
 *
 * The intermediate graph is the degree array of Sec. IV-B: deg[v] is v's degree in G - S, or
 * REMOVED when v is in S; |S| and the number of remaining edges m travel with it.
 *
 * Readings of the paper this file takes (each one is listed in the design notes):
 *   R1 Each reduction rule is applied as one simultaneous pass: every vertex that satisfies the
 *      rule in the state at the start of the pass is found, then all of the chosen vertices go
 *      into S together.  Sec. IV-D's tie-breaks decide the conflicts: of two adjacent degree-one
 *      vertices only the one with the smaller id goes into S; of several degree-two vertices in
 *      one triangle only the smallest-id one has its neighbours put into S.
 *   R2 Rule order inside the fixpoint: degree-one pass, degree-two-triangle pass, high-degree
 *      pass, repeated until a whole round changes nothing.
 *   R3 Stop check (Sec. II-B): MVC prunes when |S| >= best or m > t^2 with t = best-|S|-1;
 *      PVC prunes when |S| > k or m > t^2 with t = k-|S|.
 *   R4 The high-degree rule runs in MVC too (threshold best-|S|-1), since the edge bound of the
 *      stop check relies on it; the PVC threshold is k-|S|.
 *   R5 Greedy (Sec. II-B): repeat { degree-one and degree-two-triangle rules to a fixpoint;
 *      if edgeless stop; put the maximum-degree vertex into S }.  It has no incumbent yet, so it
 *      skips the high-degree rule.
 *   R6 PVC answers yes at once, with the greedy cover, when greedy <= k; k < 0 is always no.
 *   R7 Branch vertex: maximum current degree, ties to the lowest id.  The search visits the
 *      "take v" child before the "take N(v)" child.
 *
 * Pins (tests/test_oracle_pins.py): closed forms, brute force, Konig, complement cliques, tree
 * dynamic programme, disjoint unions, PVC around the minimum, hand-derived rule cases and greedy
 * runs.  Parity unpinned: the node counts and which minimum cover the search returns.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define REMOVED (-1)

enum { ORC_MVC = 0, ORC_PVC = 1 };
enum { RULE_DEG1 = 1, RULE_DEG2TRI = 2, RULE_HIGH = 4, RULE_ALL = 7 };

typedef struct {
    int32_t n;
    const int32_t *off; /* n+1 */
    const int32_t *adj; /* off[n] */
} graph_t;

typedef struct {
    int32_t *deg; /* n entries */
    int32_t S;    /* |S| */
    int64_t m;    /* edges of G - S */
} state_t;

/* ---------------------------------------------------------------------------------------------
 * Removing a set of vertices (Sec. IV-B): each vertex of the set gets the sentinel, each live
 * neighbour outside the set loses one degree per removed neighbour, m loses every edge that has
 * an endpoint in the set, |S| grows by the size of the set.
 * ------------------------------------------------------------------------------------------- */
static int32_t remove_marked(const graph_t *g, state_t *x, const uint8_t *mark)
{
    int32_t added = 0;
    for (int32_t v = 0; v < g->n; v++) {
        if (!mark[v]) continue;
        for (int32_t e = g->off[v]; e < g->off[v + 1]; e++) {
            int32_t u = g->adj[e];
            if (x->deg[u] == REMOVED) continue;
            if (!mark[u]) {
                x->deg[u] -= 1; /* edge vu leaves the graph */
                x->m -= 1;
            } else if (u > v) {
                x->m -= 1; /* edge between two removed vertices: count it once */
            }
        }
        added++;
    }
    for (int32_t v = 0; v < g->n; v++)
        if (mark[v]) x->deg[v] = REMOVED;
    x->S += added;
    return added;
}

static int32_t live_neighbour(const graph_t *g, const state_t *x, int32_t v, int32_t skip)
{
    for (int32_t e = g->off[v]; e < g->off[v + 1]; e++) {
        int32_t u = g->adj[e];
        if (x->deg[u] != REMOVED && u != skip) return u;
    }
    return -1;
}

static int adjacent(const graph_t *g, int32_t a, int32_t b)
{
    for (int32_t e = g->off[a]; e < g->off[a + 1]; e++)
        if (g->adj[e] == b) return 1;
    return 0;
}

/* Degree-one rule (Sec. II-B; tie-breaks of Sec. IV-D): the neighbour of a degree-one vertex goes
 * into S.  When the neighbour has degree one too (an isolated edge), only the smaller id goes. */
static int pass_degree_one(const graph_t *g, state_t *x, uint8_t *mark)
{
    int any = 0;
    memset(mark, 0, (size_t)g->n);
    for (int32_t v = 0; v < g->n; v++) {
        if (x->deg[v] != 1) continue;
        int32_t u = live_neighbour(g, x, v, -1);
        if (x->deg[u] == 1 && u > v) continue; /* isolated edge: v (smaller) is taken by u's turn */
        mark[u] = 1;
        any = 1;
    }
    if (any) remove_marked(g, x, mark);
    return any;
}

/* Degree-two-triangle rule (Sec. II-B; tie-break of Sec. IV-D): if N(v) = {u, w} and uw is an
 * edge, u and w go into S.  Only the smallest-id degree-two vertex of a triangle applies it. */
static int pass_degree_two_triangle(const graph_t *g, state_t *x, uint8_t *mark)
{
    int any = 0;
    memset(mark, 0, (size_t)g->n);
    for (int32_t v = 0; v < g->n; v++) {
        if (x->deg[v] != 2) continue;
        int32_t u = live_neighbour(g, x, v, -1);
        int32_t w = live_neighbour(g, x, v, u);
        if (!adjacent(g, u, w)) continue;
        if ((x->deg[u] == 2 && u < v) || (x->deg[w] == 2 && w < v)) continue;
        mark[u] = 1;
        mark[w] = 1;
        any = 1;
    }
    if (any) remove_marked(g, x, mark);
    return any;
}

/* High-degree rule (Sec. II-B): a vertex whose degree exceeds the threshold goes into S.
 * MVC threshold best-|S|-1, PVC threshold k-|S|. */
static int pass_high_degree(const graph_t *g, state_t *x, uint8_t *mark, int mode, int32_t bound)
{
    int32_t t = (mode == ORC_MVC) ? bound - x->S - 1 : bound - x->S;
    int any = 0;
    memset(mark, 0, (size_t)g->n);
    for (int32_t v = 0; v < g->n; v++) {
        if (x->deg[v] != REMOVED && x->deg[v] > t) {
            mark[v] = 1;
            any = 1;
        }
    }
    if (any) remove_marked(g, x, mark);
    return any;
}

/* Apply the chosen rules again and again until a whole round leaves the degree array as it was
 * (the fixpoint of Sec. II-B).  Returns the number of rounds. */
static int32_t reduce(const graph_t *g, state_t *x, uint8_t *mark, int mode, int32_t bound, int rules)
{
    int32_t rounds = 0;
    int changed;
    do {
        changed = 0;
        if (rules & RULE_DEG1) changed |= pass_degree_one(g, x, mark);
        if (rules & RULE_DEG2TRI) changed |= pass_degree_two_triangle(g, x, mark);
        if (rules & RULE_HIGH) changed |= pass_high_degree(g, x, mark, mode, bound);
        rounds++;
    } while (changed);
    return rounds;
}

/* Stop check (Sec. II-B): nonzero when no solution better than best (MVC) / within k (PVC) can
 * exist at or below this node. */
static int must_stop(const state_t *x, int mode, int32_t bound)
{
    int64_t t;
    if (mode == ORC_MVC) {
        if (x->S >= bound) return 1;
        t = (int64_t)bound - x->S - 1;
    } else {
        if (x->S > bound) return 1;
        t = (int64_t)bound - x->S;
    }
    return x->m > t * t;
}

/* Maximum current degree, ties to the lowest id (Sec. II-B and IV-B); -1 if no live vertex. */
static int32_t max_degree_vertex(const graph_t *g, const state_t *x)
{
    int32_t best_v = -1, best_d = -1;
    for (int32_t v = 0; v < g->n; v++) {
        if (x->deg[v] > best_d) {
            best_d = x->deg[v];
            best_v = v;
        }
    }
    return best_v;
}

static void init_state(const graph_t *g, state_t *x)
{
    for (int32_t v = 0; v < g->n; v++) x->deg[v] = g->off[v + 1] - g->off[v];
    x->S = 0;
    x->m = g->off[g->n] / 2;
}

static void copy_state(int32_t n, state_t *dst, const state_t *src)
{
    memcpy(dst->deg, src->deg, sizeof(int32_t) * (size_t)n);
    dst->S = src->S;
    dst->m = src->m;
}

static void write_cover(int32_t n, const state_t *x, int32_t *cover_mask)
{
    if (!cover_mask) return;
    for (int32_t v = 0; v < n; v++) cover_mask[v] = (x->deg[v] == REMOVED);
}

/* ---------------------------------------------------------------------------------------------
 * Greedy upper bound (Sec. II-B, reading R5)
 * ------------------------------------------------------------------------------------------- */
int32_t orc_greedy(int32_t n, const int32_t *off, const int32_t *adj, int32_t *cover_mask)
{
    graph_t g = {n, off, adj};
    state_t x;
    uint8_t *mark = (uint8_t *)malloc((size_t)n + 1);
    x.deg = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    init_state(&g, &x);
    for (;;) {
        reduce(&g, &x, mark, ORC_MVC, 0, RULE_DEG1 | RULE_DEG2TRI);
        if (x.m == 0) break;
        int32_t v = max_degree_vertex(&g, &x);
        memset(mark, 0, (size_t)n);
        mark[v] = 1;
        remove_marked(&g, &x, mark);
    }
    write_cover(n, &x, cover_mask);
    int32_t size = x.S;
    free(x.deg);
    free(mark);
    return size;
}

/* ---------------------------------------------------------------------------------------------
 * Branch-and-reduce search (Sec. II-B)
 * ------------------------------------------------------------------------------------------- */
typedef struct {
    const graph_t *g;
    int mode;
    int32_t bound;    /* MVC: best so far; PVC: k */
    int32_t *cover;   /* best cover so far (0/1 mask), may be NULL */
    int found;        /* PVC: a cover of size <= k was found */
    int64_t nodes;    /* tree nodes visited */
    int64_t max_nodes;
    int limit_hit;
    int32_t max_depth;
    int32_t n_levels;
    state_t *levels;  /* one state per recursion depth, allocated up front */
    uint8_t *mark;
} search_t;

static void search(search_t *s, int32_t depth)
{
    const graph_t *g = s->g;
    state_t *x = &s->levels[depth];
    if (s->found || s->limit_hit) return;
    if (s->max_nodes > 0 && s->nodes >= s->max_nodes) {
        s->limit_hit = 1;
        return;
    }
    s->nodes++;
    if (depth > s->max_depth) s->max_depth = depth;

    reduce(g, x, s->mark, s->mode, s->bound, RULE_ALL);
    if (must_stop(x, s->mode, s->bound)) return;
    if (x->m == 0) {
        if (s->mode == ORC_MVC) {
            s->bound = x->S; /* must_stop guarantees x->S < best */
        } else {
            s->found = 1;
        }
        write_cover(g->n, x, s->cover);
        return;
    }
    int32_t v = max_degree_vertex(g, x);
    state_t *child = &s->levels[depth + 1];

    /* child 1: v goes into S */
    copy_state(g->n, child, x);
    memset(s->mark, 0, (size_t)g->n);
    s->mark[v] = 1;
    remove_marked(g, child, s->mark);
    search(s, depth + 1);

    /* child 2: every live neighbour of v goes into S */
    copy_state(g->n, child, x);
    memset(s->mark, 0, (size_t)g->n);
    for (int32_t e = g->off[v]; e < g->off[v + 1]; e++)
        if (x->deg[g->adj[e]] != REMOVED) s->mark[g->adj[e]] = 1;
    remove_marked(g, child, s->mark);
    search(s, depth + 1);
}

static int run_search(search_t *s, const graph_t *g)
{
    /* Every branch puts at least one vertex into S, so depth <= n. */
    s->n_levels = g->n + 2;
    s->levels = (state_t *)calloc((size_t)s->n_levels, sizeof(state_t));
    s->mark = (uint8_t *)malloc((size_t)g->n + 1);
    if (!s->levels || !s->mark) return -1;
    for (int32_t i = 0; i < s->n_levels; i++) {
        s->levels[i].deg = (int32_t *)malloc(sizeof(int32_t) * ((size_t)g->n + 1));
        if (!s->levels[i].deg) return -1;
    }
    init_state(g, &s->levels[0]);
    search(s, 0);
    for (int32_t i = 0; i < s->n_levels; i++) free(s->levels[i].deg);
    free(s->levels);
    free(s->mark);
    return 0;
}

/* MVC.  Returns the minimum cover size (or -1 on allocation failure, -2 if max_nodes was hit);
 * cover_mask (n entries, may be NULL) receives a cover of that size; stats[0] = nodes visited,
 * stats[1] = greedy bound, stats[2] = maximum recursion depth. */
int32_t orc_mvc(int32_t n, const int32_t *off, const int32_t *adj, int32_t *cover_mask,
                int64_t max_nodes, int64_t *stats)
{
    graph_t g = {n, off, adj};
    search_t s;
    memset(&s, 0, sizeof(s));
    s.g = &g;
    s.mode = ORC_MVC;
    s.cover = cover_mask;
    s.max_nodes = max_nodes;
    int32_t u = orc_greedy(n, off, adj, cover_mask); /* incumbent = greedy cover */
    s.bound = u;
    if (run_search(&s, &g) != 0) return -1;
    if (stats) {
        stats[0] = s.nodes;
        stats[1] = u;
        stats[2] = s.max_depth;
    }
    if (s.limit_hit) return -2;
    return s.bound;
}

/* PVC.  Returns 1 (a cover of size <= k exists), 0 (none), -1 on allocation failure, -2 if
 * max_nodes was hit.  cover_mask receives the cover when the answer is 1. */
int32_t orc_pvc(int32_t n, const int32_t *off, const int32_t *adj, int32_t k, int32_t *cover_mask,
                int64_t max_nodes, int64_t *stats)
{
    graph_t g = {n, off, adj};
    search_t s;
    if (stats) stats[0] = stats[1] = stats[2] = 0;
    if (k < 0) return 0;
    int32_t *greedy_cover = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t u = orc_greedy(n, off, adj, greedy_cover);
    if (stats) stats[1] = u;
    if (u <= k) { /* reading R6 */
        if (cover_mask) memcpy(cover_mask, greedy_cover, sizeof(int32_t) * (size_t)n);
        free(greedy_cover);
        return 1;
    }
    free(greedy_cover);
    memset(&s, 0, sizeof(s));
    s.g = &g;
    s.mode = ORC_PVC;
    s.bound = k;
    s.cover = cover_mask;
    s.max_nodes = max_nodes;
    if (run_search(&s, &g) != 0) return -1;
    if (stats) {
        stats[0] = s.nodes;
        stats[2] = s.max_depth;
    }
    if (s.found) return 1;
    if (s.limit_hit) return -2;
    return 0;
}

/* One tree node's reduction, for rule tests: deg (n entries) and *S, *m are updated in place by
 * the chosen rules until a fixpoint.  mode/bound as for the search (bound = best for MVC, k for
 * PVC).  Returns 1 if the stop check then prunes the node, else 0. */
int32_t orc_reduce_node(int32_t n, const int32_t *off, const int32_t *adj, int32_t *deg,
                        int32_t *S, int64_t *m, int32_t mode, int32_t bound, int32_t rules)
{
    graph_t g = {n, off, adj};
    state_t x = {deg, *S, *m};
    uint8_t *mark = (uint8_t *)malloc((size_t)n + 1);
    reduce(&g, &x, mark, mode, bound, rules);
    free(mark);
    *S = x.S;
    *m = x.m;
    return must_stop(&x, mode, bound);
}
