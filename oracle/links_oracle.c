/*
 * links_oracle.c -- plain, slow, FP64 reference of the linkage-simulation hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load it.  The product library neither links nor
 * calls it, and the two share no code, header, table or constant.
 *
 * Built with -O2 -ffp-contract=off: every operation is a separately rounded IEEE
 * double operation in the order written here (no fused multiply-add).
 *
 * What it computes, and where the paper defines it (LINKS, arXiv 2208.14567):
 *   - mechanism representation: n x n adjacency A, per-joint type (0 fixed,
 *     1 simple, 2 actuated) and initial positions (Sec. "Mechanism
 *     Representation"; Sec. "Dataset Features & Statistics", item Mechanisms);
 *   - solve order (Sec. "Graphical Simulator", Fig. "solver"): starting from the
 *     known joints (fixed + actuated), repeatedly solve a joint with two known
 *     neighbours; fail on complex loops;
 *   - 1-DOF check from the mobility equation (Eq. 1) and the J-operator argument
 *     (Sec. "1-DOF Operator"): every simple joint consumes exactly two links;
 *   - simulation over T equally spaced actuator positions of one full turn
 *     (Sec. "Dataset Features & Statistics", item Simulation Data) with the locking test
 *     (Sec. "Finding Valid Initial Positions", Infeasibility rule);
 *   - path normalisation (centroid, unit RMS radius, principal axis on +x) and
 *     the bidirectional chamfer distance (Sec. "A Case Study of Mechanism
 *     Retrieval").
 *
 * Readings where the paper is silent:
 *   - the crank pivot is the lowest-index fixed neighbour of the actuated joint;
 *   - among unknown joints with >= 2 known neighbours, the lowest index is solved
 *     first; its two known neighbours are its parents i < j; > 2 known
 *     neighbours is over-constraint;
 *   - branch: the orientation sign s = sgn((p_j - p_i) x (p_k - p_i)) of the
 *     initial configuration is kept for all steps (0 counts as +1);
 *   - step t uses crank angle 2*pi*t/T, counter-clockwise from the initial crank;
 *   - a dyad with q = D / (4 r1^2 r2^2) not > 0 locks the mechanism at that step
 *     (D = 4 d^2 r1^2 - e^2 is 16 x the squared triangle area; q is the squared
 *     sine of the angle at the solved joint); trajectories are NaN from the
 *     locking step on;
 *   - min_disc = min of q over all dyads of the steps before the lock.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define LO_MAXJ 64

enum {
    LO_OK = 0,
    LO_BAD_SIZE = 1,
    LO_BAD_TYPE = 2,
    LO_BAD_ADJ = 3,
    LO_NO_MOTOR = 4,
    LO_NO_PIVOT = 5,
    LO_NOT_DYAD_SOLVABLE = 6,
    LO_OVERCONSTRAINED = 7
};

typedef struct {
    int32_t status, n, motor, pivot, n_dyads, coupler;
    int32_t k[LO_MAXJ], i[LO_MAXJ], j[LO_MAXJ], s[LO_MAXJ];
    double r1sq[LO_MAXJ], r2sq[LO_MAXJ];
} lo_plan_t;

static double sq_dist(const double* a, const double* b) {
    double dx = a[0] - b[0];
    double dy = a[1] - b[1];
    return dx * dx + dy * dy;
}

/* Solve order of one mechanism.  adj is n_max x n_max (row-major), type and pos
 * have n_max rows; only the first n joints are read. */
int lo_plan(int n, int n_max, const uint8_t* adj, const int8_t* type, const double* pos,
            lo_plan_t* P) {
    memset(P, 0, sizeof(*P));
    P->n = n;
    P->motor = P->pivot = P->coupler = -1;
    if (n < 2 || n > n_max || n_max > LO_MAXJ) return P->status = LO_BAD_SIZE;
    for (int a = 0; a < n; ++a)
        if (type[a] < 0 || type[a] > 2) return P->status = LO_BAD_TYPE;
    for (int a = 0; a < n; ++a) {
        if (adj[a * n_max + a] != 0) return P->status = LO_BAD_ADJ;
        for (int b = 0; b < n; ++b)
            if ((adj[a * n_max + b] != 0) != (adj[b * n_max + a] != 0)) return P->status = LO_BAD_ADJ;
    }
    int motor = -1, n_motor = 0;
    for (int a = 0; a < n; ++a)
        if (type[a] == 2) { motor = a; ++n_motor; }
    if (n_motor != 1) return P->status = LO_NO_MOTOR;
    int pivot = -1;
    for (int a = 0; a < n && pivot < 0; ++a)
        if (type[a] == 0 && adj[motor * n_max + a]) pivot = a;
    if (pivot < 0) return P->status = LO_NO_PIVOT;
    P->motor = motor;
    P->pivot = pivot;

    int known[LO_MAXJ];
    int n_unknown = 0, n_simple = 0;
    for (int a = 0; a < n; ++a) {
        known[a] = (type[a] != 1);
        if (!known[a]) { ++n_unknown; ++n_simple; }
    }
    int nd = 0;
    while (n_unknown > 0) {
        int pick = -1, cnt = 0;
        for (int a = 0; a < n; ++a) {
            if (known[a]) continue;
            cnt = 0;
            for (int b = 0; b < n; ++b)
                if (known[b] && adj[a * n_max + b]) ++cnt;
            if (cnt >= 2) { pick = a; break; }
        }
        if (pick < 0) return P->status = LO_NOT_DYAD_SOLVABLE;
        if (cnt > 2) return P->status = LO_OVERCONSTRAINED;
        int par[2], m = 0;
        for (int b = 0; b < n; ++b)
            if (known[b] && adj[pick * n_max + b]) par[m++] = b;
        int i = par[0], j = par[1];
        const double* pi = pos + 2 * i;
        const double* pj = pos + 2 * j;
        const double* pk = pos + 2 * pick;
        double cross = (pj[0] - pi[0]) * (pk[1] - pi[1]) - (pj[1] - pi[1]) * (pk[0] - pi[0]);
        P->k[nd] = pick;
        P->i[nd] = i;
        P->j[nd] = j;
        P->s[nd] = cross < 0.0 ? -1 : 1;
        P->r1sq[nd] = sq_dist(pk, pi);
        P->r2sq[nd] = sq_dist(pk, pj);
        ++nd;
        known[pick] = 1;
        --n_unknown;
    }
    /* 1-DOF edge count: links other than ground-ground links and the crank must be
     * exactly two per simple joint (Eq. 1 with one actuator and no redundancy). */
    int links = 0;
    for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b) {
            if (!adj[a * n_max + b]) continue;
            if (type[a] == 0 && type[b] == 0) continue;
            if ((a == motor && b == pivot) || (b == motor && a == pivot)) continue;
            ++links;
        }
    if (links != 2 * n_simple) return P->status = LO_OVERCONSTRAINED;
    P->n_dyads = nd;
    P->coupler = nd > 0 ? P->k[nd - 1] : motor;
    return P->status = LO_OK;
}

/* Joint positions at crank angle theta.  out is n_max x 2.  Returns 1 if some dyad
 * locks (then *q_lock holds its q and later dyads are NaN), else 0.  *q_min is the
 * smallest q over the dyads evaluated, *q_abs_min the smallest |q|. */
int lo_solve_at(const lo_plan_t* P, int n_max, const double* pos0, double theta, double* out,
                double* q_min, double* q_abs_min, double* q_lock) {
    const double nan = NAN;
    for (int a = 0; a < n_max; ++a) { out[2 * a] = nan; out[2 * a + 1] = nan; }
    for (int a = 0; a < P->n; ++a) {
        /* fixed joints stay put; simple joints are overwritten below */
        out[2 * a] = pos0[2 * a];
        out[2 * a + 1] = pos0[2 * a + 1];
    }
    double c = cos(theta), s = sin(theta);
    const double* pv = pos0 + 2 * P->pivot;
    double ux = pos0[2 * P->motor] - pv[0];
    double uy = pos0[2 * P->motor + 1] - pv[1];
    out[2 * P->motor] = pv[0] + (c * ux - s * uy);
    out[2 * P->motor + 1] = pv[1] + (s * ux + c * uy);
    for (int d = 0; d < P->n_dyads; ++d) {
        out[2 * P->k[d]] = nan;
        out[2 * P->k[d] + 1] = nan;
    }
    double qmin = INFINITY, qabs = INFINITY;
    for (int d = 0; d < P->n_dyads; ++d) {
        const double* pi = out + 2 * P->i[d];
        const double* pj = out + 2 * P->j[d];
        double dx = pj[0] - pi[0];
        double dy = pj[1] - pi[1];
        double d2 = dx * dx + dy * dy;
        double e = d2 + P->r1sq[d] - P->r2sq[d];
        double D = 4.0 * d2 * P->r1sq[d] - e * e;
        double q = D / (4.0 * P->r1sq[d] * P->r2sq[d]);
        double aq = fabs(q);
        if (aq < qabs || aq != aq) qabs = aq;
        if (!(q > 0.0)) {
            if (q_min) *q_min = qmin;
            if (q_abs_min) *q_abs_min = qabs;
            if (q_lock) *q_lock = q;
            return 1;
        }
        if (q < qmin) qmin = q;
        double h = sqrt(D);
        double sh = (double)P->s[d] * h;
        double inv = 1.0 / (2.0 * d2);
        out[2 * P->k[d]] = pi[0] + (e * dx - sh * dy) * inv;
        out[2 * P->k[d] + 1] = pi[1] + (e * dy + sh * dx) * inv;
    }
    if (q_min) *q_min = qmin;
    if (q_abs_min) *q_abs_min = qabs;
    if (q_lock) *q_lock = NAN;
    return 0;
}

/* Plan + simulate mechanisms [b0, b1).  Array strides follow the batch layout
 * (adj [B,n_max,n_max], type [B,n_max], pos [B,n_max,2]).  traj [B,n_max,T,2] and
 * path [B,T,2] may be NULL. */
void lo_simulate(int64_t b0, int64_t b1, int n_max, const int32_t* n_joints, const uint8_t* adj,
                 const int8_t* type, const double* pos, int T, double* traj, double* path,
                 uint8_t* valid, int16_t* lock_step, double* min_disc, double* min_abs_q,
                 int32_t* status) {
    double cur[2 * LO_MAXJ];
    lo_plan_t P;
    const double nan = NAN;
    for (int64_t b = b0; b < b1; ++b) {
        const double* p0 = pos + (size_t)b * n_max * 2;
        int st = lo_plan(n_joints[b], n_max, adj + (size_t)b * n_max * n_max, type + (size_t)b * n_max,
                         p0, &P);
        double* tr = traj ? traj + (size_t)b * n_max * T * 2 : 0;
        double* pa = path ? path + (size_t)b * T * 2 : 0;
        if (tr) for (size_t x = 0; x < (size_t)n_max * T * 2; ++x) tr[x] = nan;
        if (pa) for (size_t x = 0; x < (size_t)T * 2; ++x) pa[x] = nan;
        status[b] = st;
        if (st != LO_OK) {
            valid[b] = 0;
            lock_step[b] = -2;
            min_disc[b] = nan;
            min_abs_q[b] = nan;
            continue;
        }
        int lock = -1;
        double qmin_all = INFINITY, qabs_all = INFINITY;
        for (int t = 0; t < T; ++t) {
            double theta = 2.0 * M_PI * (double)t / (double)T;
            double qmin, qabs, qlock;
            int locked = lo_solve_at(&P, n_max, p0, theta, cur, &qmin, &qabs, &qlock);
            if (qabs < qabs_all || qabs != qabs) qabs_all = qabs;
            if (locked) { lock = t; break; }
            if (qmin < qmin_all) qmin_all = qmin;
            for (int a = 0; a < P.n; ++a)
                if (tr) {
                    tr[((size_t)a * T + t) * 2] = cur[2 * a];
                    tr[((size_t)a * T + t) * 2 + 1] = cur[2 * a + 1];
                }
            if (pa) {
                pa[2 * t] = cur[2 * P.coupler];
                pa[2 * t + 1] = cur[2 * P.coupler + 1];
            }
        }
        valid[b] = lock < 0;
        lock_step[b] = (int16_t)lock;
        min_disc[b] = qmin_all;
        min_abs_q[b] = qabs_all;
    }
}

/* Normalise curves [m0, m1) of T points (in/out [M,T,2]): centroid to the origin,
 * unit RMS radius, principal axis of the 2x2 covariance onto +x, and of the two
 * rotations that do that, the one with sum(x^3) >= 0.  An isotropic covariance
 * (lambda1 - lambda2 <= 1e-9 (lambda1 + lambda2)) is not rotated.  A curve of
 * identical points maps to zeros. */
void lo_normalize(int64_t m0, int64_t m1, int T, const double* in, double* out) {
    for (int64_t m = m0; m < m1; ++m) {
        const double* p = in + (size_t)m * T * 2;
        double* o = out + (size_t)m * T * 2;
        double cx = 0.0, cy = 0.0;
        for (int t = 0; t < T; ++t) { cx += p[2 * t]; cy += p[2 * t + 1]; }
        cx /= T;
        cy /= T;
        double r2 = 0.0;
        for (int t = 0; t < T; ++t) {
            double x = p[2 * t] - cx, y = p[2 * t + 1] - cy;
            r2 += x * x + y * y;
        }
        double rms = sqrt(r2 / T);
        if (!(rms > 0.0)) {
            for (int t = 0; t < 2 * T; ++t) o[t] = 0.0;
            continue;
        }
        double sxx = 0.0, sxy = 0.0, syy = 0.0;
        for (int t = 0; t < T; ++t) {
            double x = (p[2 * t] - cx) / rms, y = (p[2 * t + 1] - cy) / rms;
            sxx += x * x;
            sxy += x * y;
            syy += y * y;
        }
        sxx /= T;
        sxy /= T;
        syy /= T;
        double gap = sqrt((sxx - syy) * (sxx - syy) + 4.0 * sxy * sxy);
        double phi = 0.0;
        if (gap > 1e-9 * (sxx + syy)) phi = 0.5 * atan2(2.0 * sxy, sxx - syy);
        double c = cos(phi), s = sin(phi);
        double s3 = 0.0;
        for (int t = 0; t < T; ++t) {
            double x = (p[2 * t] - cx) / rms, y = (p[2 * t + 1] - cy) / rms;
            double xr = c * x + s * y;
            double yr = -s * x + c * y;
            o[2 * t] = xr;
            o[2 * t + 1] = yr;
            s3 += xr * xr * xr;
        }
        if (s3 < 0.0)
            for (int t = 0; t < 2 * T; ++t) o[t] = -o[t];
    }
}

/* The paper's path normalisation (Sec. "Dataset Curation & Processing"): find the line of
 * maximum distance between two points of the path, rotate the path so that this line is
 * horizontal, scale it so that the line has length 1, and centre the path in the unit
 * box.  Readings: the line joins the pair (a, b), a < b, of largest distance, the first
 * such pair in (a, b) order on ties; the rotation takes p_b - p_a onto +x; "centre" puts
 * the centre of the bounding box at (0.5, 0.5); a path of equal points becomes (0.5, 0.5)
 * everywhere.  If pair_in is not NULL it gives the pair to use instead of the search
 * (to compare with a computation whose float rounding picked a near-tied pair).
 * pair_out [2] and circ_var (the population variance of the distances of the normalised
 * points from (0.5, 0.5), the paper's circle statistic) may be NULL. */
void lo_normalize_maxline(int T, const double* p, double* o, const int32_t* pair_in, int32_t* pair_out,
                          double* circ_var) {
    int a = 0, b = T > 1 ? 1 : 0;
    if (pair_in) {
        a = pair_in[0];
        b = pair_in[1];
    } else {
        double best = -1.0;
        for (int u = 0; u < T; ++u)
            for (int v = u + 1; v < T; ++v) {
                double d = sq_dist(p + 2 * u, p + 2 * v);
                if (d > best) { best = d; a = u; b = v; }
            }
    }
    if (pair_out) { pair_out[0] = a; pair_out[1] = b; }
    double dx = p[2 * b] - p[2 * a], dy = p[2 * b + 1] - p[2 * a + 1];
    double d = sqrt(dx * dx + dy * dy);
    if (!(d > 0.0)) {
        for (int t = 0; t < T; ++t) { o[2 * t] = 0.5; o[2 * t + 1] = 0.5; }
        if (circ_var) *circ_var = 0.0;
        return;
    }
    double c = dx / d, s = dy / d;  /* rotation by minus the line's angle, and 1/d scale */
    double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (int t = 0; t < T; ++t) {
        double x = p[2 * t] - p[2 * a], y = p[2 * t + 1] - p[2 * a + 1];
        double xr = (c * x + s * y) / d, yr = (-s * x + c * y) / d;
        o[2 * t] = xr;
        o[2 * t + 1] = yr;
        if (xr < x0) x0 = xr;
        if (xr > x1) x1 = xr;
        if (yr < y0) y0 = yr;
        if (yr > y1) y1 = yr;
    }
    double sx = 0.5 - 0.5 * (x0 + x1), sy = 0.5 - 0.5 * (y0 + y1);
    double m = 0.0, m2 = 0.0;
    for (int t = 0; t < T; ++t) {
        o[2 * t] += sx;
        o[2 * t + 1] += sy;
        double r = sqrt((o[2 * t] - 0.5) * (o[2 * t] - 0.5) + (o[2 * t + 1] - 0.5) * (o[2 * t + 1] - 0.5));
        m += r;
        m2 += r * r;
    }
    m /= T;
    if (circ_var) *circ_var = m2 / T - m * m;
}

/* Bidirectional chamfer distance: mean over P of the Euclidean distance to the
 * nearest point of Q, plus the same from Q to P. */
double lo_chamfer(int tp, const double* P, int tq, const double* Q) {
    double sp = 0.0, sq = 0.0;
    for (int a = 0; a < tp; ++a) {
        double best = INFINITY;
        for (int b = 0; b < tq; ++b) {
            double d = sqrt(sq_dist(P + 2 * a, Q + 2 * b));
            if (d < best) best = d;
        }
        sp += best;
    }
    for (int b = 0; b < tq; ++b) {
        double best = INFINITY;
        for (int a = 0; a < tp; ++a) {
            double d = sqrt(sq_dist(Q + 2 * b, P + 2 * a));
            if (d < best) best = d;
        }
        sq += best;
    }
    return sp / tp + sq / tq;
}

/* Chamfer distance from one query curve to database curves [m0, m1) (db [M,T,2]). */
void lo_chamfer_many(int tq, const double* q, int64_t m0, int64_t m1, int T, const double* db,
                     double* out) {
    for (int64_t m = m0; m < m1; ++m) out[m] = lo_chamfer(tq, q, T, db + (size_t)m * T * 2);
}
