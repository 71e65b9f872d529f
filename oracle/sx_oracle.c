/*
 * sx_oracle.c -- plain FP64 CPU reference of the SimpleX2 direction-conserving
 * transport (DCT) sweep.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the CPU-baseline leg of the benchmark call it; the product path never
 * does.  It shares no code with the CUDA library.
 *
 * It follows the paper (Paardekooper, Kruip & Icke 2010, "SimpleX2") step by
 * step, slowly and in the obvious order:
 *
 *   Sect. 2.2    interaction at a vertex: N_abs = N_in (1 - e^-tau), N_out = N_in e^-tau
 *   Sect. 2.2.3  direction-conserving transport: photons live in n global
 *                direction bins; a bin is associated with a Delaunay edge of
 *                the vertex and its photons are split over the d = 3 most
 *                straightforward neighbours of that edge (none beyond 90 deg);
 *                the bins are rotated at random between steps; a global factor
 *                corrects the zig-zag path length.
 *   Sect. 4.4    Eq. (optical_depth): dtau = n_HI sigma dL (sigma restored).
 *   Sect. 4.5    Eqs. (rate_eq_subcycle, phot_ion_rate_subcycle): the rate
 *                equation is subcycled at constant ionising flux, photon
 *                conserving; once equilibrium is reached the last subcycle's
 *                values are kept for the rest of the step.
 *   Sect. 4.6    photons move one Delaunay edge per radiative-transfer step.
 *   Sect. 2.2.2  ballistic transport: photons that came in along an edge go
 *                on, in d = 3 equal parts, to the most straightforward
 *                neighbours with respect to that incoming direction (none
 *                beyond 90 deg); a source sends to all its neighbours.
 *   Sect. 2.2.4  combined transport: ballistic where the optical depth is
 *                high, direction conserving where it is low; photons change
 *                representation (bins <-> edges) on arrival.
 *   Sect. 2.2.1, 4.5  diffuse recombination radiation (optional; the paper's
 *                tests use the on-the-spot approximation instead): case A
 *                recombination, and every recombination straight to the
 *                ground level emits an ionising photon that leaves its cell
 *                with no memory of direction, so every ionised cell is a
 *                source.
 *
 * Readings of points the paper leaves open (all listed in the design notes):
 *   - association: bin b of vertex i goes with the edge k maximising the dot
 *     product of int-quantised unit vectors (Q = 127), ties -> lowest slot;
 *   - straight[i][k]: the <= 3 slots k' with the largest positive quantised
 *     dot with edge k (k itself included), ties -> lowest slot;
 *   - random rotation: Philox4x32-10 (Salmon et al. 2011) with key = seed and
 *     counter = (step lo, step hi, attempt, tag); four uniforms in (-1,1),
 *     accepted inside the unit 4-ball, give a uniform quaternion; the
 *     rotation matrix is its polynomial form divided by |q|^2;
 *   - a rotation moves every packet in flight to the bin of the new
 *     orientation closest to its old bin (photons keep their direction);
 *   - path correction kappa = sum(progress along the bin) / sum(edge length)
 *     over interior vertices and unrotated bins; dL_i = kappa * mean edge length;
 *   - subcycle length h = min(t_left, f_c / (Gamma + R)); equilibrium when
 *     |dy| <= tol * y after a subcycle; cap max_sub subcycles;
 *   - sinks (boundary shell) absorb everything into "escaped";
 *   - ballistic straight set of the in-edge from u: the <= 3 slots k with the
 *     largest positive quantised dot q_ik . (-q_iu), ties -> lowest slot;
 *   - combined: a vertex is ballistic in a step when y tau_max >= tau_switch
 *     with y its neutral fraction at the start of the step; it keeps its
 *     photons per in-edge (bins arriving along an edge summed into it), a
 *     direction-conserving vertex keeps bins (a packet arriving along an edge
 *     goes to the bin closest to the direction it travelled);
 *   - a ballistic source sends its photons in equal parts along all edges;
 *   - diffuse radiation: the recombinations of a step are summed over its
 *     subcycles (the hold after equilibrium at the last subcycle's rate); a
 *     fraction (alpha_A - alpha_B) / alpha_A of them emit one photon each; a
 *     cell's photons of one step enter in the next step, after the sources'
 *     photons and as a source's photons do (the cell absorbs first): an
 *     equal share in every bin at a direction-conserving vertex, the
 *     vertex's own photons, sent to all neighbours in equal parts, at a
 *     ballistic one.
 *
 * Build: cc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared
 * (-ffp-contract=off keeps every a*b+c a separate multiply and add so that the
 * quantised directions are the IEEE results of the stated operations).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OX_Q 127.0
#define OX_MAX_STRAIGHT 3
#define OX_ROT_TAG 0x53583252u /* "SX2R" */
#define OX_ROT_MAX_ATTEMPTS 64

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (Salmon et al. 2011).       */
/* ------------------------------------------------------------------------ */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void ox_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(M0, c0, &hi0, &lo0);
        mulhilo32(M1, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Random rotation of the direction bins for step `step` (Sect. 2.2.3).      */
/* Returns the number of Philox draws used (1..64); R row-major.             */
/* ------------------------------------------------------------------------ */
int ox_rotation(uint64_t seed, int64_t step, double R[9]) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t s = (uint64_t)step;
    for (int a = 0; a < OX_ROT_MAX_ATTEMPTS; ++a) {
        uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(s >> 32), (uint32_t)a, OX_ROT_TAG};
        uint32_t x[4];
        ox_philox4x32_10(ctr, key, x);
        double v[4];
        for (int i = 0; i < 4; ++i) v[i] = ((double)(int32_t)x[i] + 0.5) * 0x1p-31;
        double w = v[0], qx = v[1], qy = v[2], qz = v[3];
        double ww = w * w, xx = qx * qx, yy = qy * qy, zz = qz * qz;
        double n2 = ((ww + xx) + yy) + zz;
        if (!(n2 <= 1.0)) continue;
        double xy = qx * qy, xz = qx * qz, yz = qy * qz;
        double wx = w * qx, wy = w * qy, wz = w * qz;
        R[0] = (((ww + xx) - yy) - zz) / n2;
        R[1] = ((xy - wz) * 2.0) / n2;
        R[2] = ((xz + wy) * 2.0) / n2;
        R[3] = ((xy + wz) * 2.0) / n2;
        R[4] = (((ww - xx) + yy) - zz) / n2;
        R[5] = ((yz - wx) * 2.0) / n2;
        R[6] = ((xz - wy) * 2.0) / n2;
        R[7] = ((yz + wx) * 2.0) / n2;
        R[8] = (((ww - xx) - yy) + zz) / n2;
        return a + 1;
    }
    for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
    return OX_ROT_MAX_ATTEMPTS;
}

static int quantise(double u) {
    double r = rint(OX_Q * u);
    if (r > OX_Q) r = OX_Q;
    if (r < -OX_Q) r = -OX_Q;
    return (int)r;
}

/* Quantised rotated bins: q[b] = rint(127 * (R d_b)). */
void ox_rotated_bins(const double R[9], int nbins, const double *bins, int32_t *q) {
    for (int b = 0; b < nbins; ++b) {
        const double *d = bins + 3 * b;
        for (int r = 0; r < 3; ++r) {
            double u = (R[3 * r] * d[0] + R[3 * r + 1] * d[1]) + R[3 * r + 2] * d[2];
            q[3 * b + r] = quantise(u);
        }
    }
}

/* Orientation change between steps (Sect. 2.2.3): a packet in bin b of the old
 * orientation keeps its direction by moving to the new bin closest to it,
 * map[b] = argmax_b' q_new[b'] . q_old[b] (exact integers, ties -> lowest b'). */
void ox_bin_map(int nbins, const int32_t *q_old, const int32_t *q_new, int32_t *map) {
    for (int b = 0; b < nbins; ++b) {
        int best = 0;
        int64_t bestd = 0;
        for (int b2 = 0; b2 < nbins; ++b2) {
            int64_t d = (int64_t)q_new[3 * b2] * q_old[3 * b] + (int64_t)q_new[3 * b2 + 1] * q_old[3 * b + 1] +
                        (int64_t)q_new[3 * b2 + 2] * q_old[3 * b + 2];
            if (b2 == 0 || d > bestd) {
                best = b2;
                bestd = d;
            }
        }
        map[b] = best;
    }
}

/* Quantised unit vector of edge i -> k. */
static void edge_q(const double *pi, const double *pk, int32_t q[3], double *len_out) {
    double dx = pk[0] - pi[0], dy = pk[1] - pi[1], dz = pk[2] - pi[2];
    double len = sqrt((dx * dx + dy * dy) + dz * dz);
    q[0] = quantise(dx / len);
    q[1] = quantise(dy / len);
    q[2] = quantise(dz / len);
    if (len_out) *len_out = len;
}

static int64_t idot(const int32_t *a, const int32_t *b) {
    return (int64_t)a[0] * b[0] + (int64_t)a[1] * b[1] + (int64_t)a[2] * b[2];
}

/* ------------------------------------------------------------------------ */
/* Per-edge tables (Sect. 2.2.2: most straightforward neighbours, computed   */
/* once per grid).                                                           */
/* ------------------------------------------------------------------------ */
void ox_edge_tables(int64_t n, const double *pos, const int64_t *row_ptr, const int32_t *col,
                    int32_t *qedge /* nnz*3 */, uint8_t *straight /* nnz*4: 3 slots + count */,
                    double *mean_len /* n */) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t r0 = row_ptr[i], r1 = row_ptr[i + 1];
        double sum = 0.0;
        for (int64_t e = r0; e < r1; ++e) {
            double len;
            edge_q(pos + 3 * i, pos + 3 * (int64_t)col[e], qedge + 3 * e, &len);
            sum += len;
        }
        mean_len[i] = (r1 > r0) ? sum / (double)(r1 - r0) : 0.0;
        for (int64_t e = r0; e < r1; ++e) {
            int64_t best[OX_MAX_STRAIGHT];
            int slot[OX_MAX_STRAIGHT];
            int cnt = 0;
            for (int64_t e2 = r0; e2 < r1; ++e2) {
                int64_t d = idot(qedge + 3 * e, qedge + 3 * e2);
                if (d <= 0) continue;
                int k2 = (int)(e2 - r0);
                /* insert keeping descending dot; equal dots keep the earlier slot first */
                int pos_ins = cnt;
                while (pos_ins > 0 && d > best[pos_ins - 1]) pos_ins--;
                if (pos_ins >= OX_MAX_STRAIGHT) continue;
                int last = cnt < OX_MAX_STRAIGHT ? cnt : OX_MAX_STRAIGHT - 1;
                for (int m = last; m > pos_ins; --m) {
                    best[m] = best[m - 1];
                    slot[m] = slot[m - 1];
                }
                best[pos_ins] = d;
                slot[pos_ins] = k2;
                if (cnt < OX_MAX_STRAIGHT) cnt++;
            }
            for (int m = 0; m < OX_MAX_STRAIGHT; ++m)
                straight[4 * e + m] = (m < cnt) ? (uint8_t)slot[m] : 0xFF;
            straight[4 * e + 3] = (uint8_t)cnt;
        }
    }
}

/* Association of one bin at vertex i: argmax_k q_b . q_ik, ties -> lowest k. */
static int associate(const int32_t *qb, const int32_t *qedge, int64_t r0, int64_t r1) {
    int best = -1;
    int64_t bestd = 0;
    for (int64_t e = r0; e < r1; ++e) {
        int64_t d = idot(qb, qedge + 3 * e);
        if (best < 0 || d > bestd) {
            best = (int)(e - r0);
            bestd = d;
        }
    }
    return best;
}

/* Global path-length correction factor (Sect. 2.2.3, Fig. photon_path). */
double ox_kappa(int64_t n, const double *pos, const int64_t *row_ptr, const int32_t *col,
                const uint8_t *flags, const int32_t *qedge, const uint8_t *straight, int nbins,
                const double *bins) {
    int32_t *qb = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)nbins);
    const double I3[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    ox_rotated_bins(I3, nbins, bins, qb);
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (flags[i] & 1) continue;
        int64_t r0 = row_ptr[i], r1 = row_ptr[i + 1];
        if (r1 == r0) continue;
        for (int b = 0; b < nbins; ++b) {
            int k = associate(qb + 3 * b, qedge, r0, r1);
            const uint8_t *st = straight + 4 * (r0 + k);
            int cnt = st[3];
            if (cnt == 0) continue;
            double prog = 0.0, path = 0.0;
            for (int m = 0; m < cnt; ++m) {
                int64_t j = col[r0 + st[m]];
                double dx = pos[3 * j] - pos[3 * i], dy = pos[3 * j + 1] - pos[3 * i + 1],
                       dz = pos[3 * j + 2] - pos[3 * i + 2];
                const double *d = bins + 3 * b;
                prog += (dx * d[0] + dy * d[1]) + dz * d[2];
                path += sqrt((dx * dx + dy * dy) + dz * dz);
            }
            num += prog / cnt;
            den += path / cnt;
        }
    }
    free(qb);
    return den > 0.0 ? num / den : 1.0;
}

/* ------------------------------------------------------------------------ */
/* Photoionisation / recombination of one cell over one transfer step        */
/* (Sect. 4.5, Eqs. rate_eq_subcycle and phot_ion_rate_subcycle).            */
/*   y       neutral fraction (1 - x), updated in place                      */
/*   N_in    photons entering the cell during the step                       */
/*   A       hydrogen atoms in the cell, n_H V                               */
/*   tau_max optical depth of the fully neutral cell, n_H sigma dL           */
/*   R0      alpha_B n_H (recombinations per ion per second at x = 1)        */
/* Returns the transmitted fraction f = (1/dt) sum_k e^{-tau_k} h_k, so that */
/* N_out = f N_in and N_abs = (1 - f) N_in.                                  */
/* ------------------------------------------------------------------------ */
/* rec_out (may be NULL): recombinations per atom during the step,         */
/* sum_k R0 x_k^2 h_k (the hold after equilibrium at the last subcycle's     */
/* rate).                                                                    */
double ox_chem_rec(double *y_io, double N_in, double dt, double A, double tau_max, double R0,
                   double fc, double tol, int max_sub, int *nsub_out, int *capped_out,
                   double *rec_out) {
    double y = *y_io;
    if (rec_out) *rec_out = 0.0;
    if (!(A > 0.0)) {              /* no atoms (n_H = 0): tau = 0, the cell is transparent */
        if (nsub_out) *nsub_out = 0;
        if (capped_out) *capped_out = 0;
        return 1.0;
    }
    double rec_int = 0.0;          /* integral of R0 x^2 dt */
    double F = N_in / dt;          /* photons per second, constant over the step */
    double t_left = dt;
    double trans_int = 0.0;        /* integral of e^{-tau} dt */
    int nsub = 0, capped = 0;
    while (t_left > 0.0) {
        double tau = tau_max * y;
        double tr = exp(-tau);               /* transmitted fraction */
        double ab = -expm1(-tau);            /* absorbed fraction */
        double ion = F * ab / A;             /* photoionisations per atom per second (= Gamma y) */
        double x = 1.0 - y;
        double rec = R0 * x * x;             /* recombinations per atom per second */
        double gam = (y > 0.0) ? ion / y : F * tau_max / A;  /* Gamma per neutral atom */
        double rate = gam + R0 * x;          /* 1 / (equilibration time) */
        double h = t_left;
        if (rate > 0.0) {
            double hc = fc / rate;
            if (hc < h) h = hc;
        }
        double y_new = y + (rec - ion) * h;
        trans_int += tr * h;
        rec_int += rec * h;
        t_left = (h == t_left) ? 0.0 : t_left - h;
        nsub++;
        int eq = fabs(y_new - y) <= tol * y_new;
        y = y_new;
        if (t_left > 0.0 && (eq || nsub >= max_sub)) {
            /* equilibrium (or cap): keep the last subcycle's values */
            if (!eq) capped = 1;
            trans_int += tr * t_left;
            rec_int += rec * t_left;
            t_left = 0.0;
        }
    }
    *y_io = y;
    if (nsub_out) *nsub_out = nsub;
    if (capped_out) *capped_out = capped;
    if (rec_out) *rec_out = rec_int;
    return trans_int / dt;
}

double ox_chem(double *y_io, double N_in, double dt, double A, double tau_max, double R0,
               double fc, double tol, int max_sub, int *nsub_out, int *capped_out) {
    return ox_chem_rec(y_io, N_in, dt, A, tau_max, R0, fc, tol, max_sub, nsub_out, capped_out, NULL);
}

/* ------------------------------------------------------------------------ */
/* Ballistic transport (Sect. 2.2.2): photons that came in along edge u -> i */
/* go on in p = d = 3 equal parts to the most straightforward neighbours of  */
/* i with respect to the direction they travelled (the edge i -> u           */
/* reversed); neighbours beyond 90 degrees are left out.                     */
/*   stb[e]: for the in-edge of slot j of vertex i, the <= 3 slots k with    */
/*   the largest positive quantised dot q_ik . (-q_ij), ties -> lowest slot; */
/*   twin[e]: the index of edge i -> k in k's row (rows ascending).          */
/* ------------------------------------------------------------------------ */
void ox_ballistic_tables(int64_t n, const int64_t *row_ptr, const int32_t *col,
                         const int32_t *qedge, uint8_t *stb /* nnz*4 */, int64_t *twin /* nnz */) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t r0 = row_ptr[i], r1 = row_ptr[i + 1];
        for (int64_t e = r0; e < r1; ++e) {
            int32_t back[3] = {-qedge[3 * e], -qedge[3 * e + 1], -qedge[3 * e + 2]};
            int64_t best[OX_MAX_STRAIGHT];
            int slot[OX_MAX_STRAIGHT];
            int cnt = 0;
            for (int64_t e2 = r0; e2 < r1; ++e2) {
                int64_t d = idot(back, qedge + 3 * e2);
                if (d <= 0) continue;
                /* keep the first three in (dot descending, slot ascending) order */
                int at = cnt;
                while (at > 0 && d > best[at - 1]) at--;
                if (at >= OX_MAX_STRAIGHT) continue;
                int last = cnt < OX_MAX_STRAIGHT ? cnt : OX_MAX_STRAIGHT - 1;
                for (int m = last; m > at; --m) {
                    best[m] = best[m - 1];
                    slot[m] = slot[m - 1];
                }
                best[at] = d;
                slot[at] = (int)(e2 - r0);
                if (cnt < OX_MAX_STRAIGHT) cnt++;
            }
            for (int m = 0; m < OX_MAX_STRAIGHT; ++m) stb[4 * e + m] = (m < cnt) ? (uint8_t)slot[m] : 0xFF;
            stb[4 * e + 3] = (uint8_t)cnt;
            int64_t k = col[e], lo = row_ptr[k], hi = row_ptr[k + 1] - 1, t = -1;
            while (lo <= hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (col[mid] == (int32_t)i) {
                    t = mid;
                    break;
                }
                if (col[mid] < (int32_t)i) lo = mid + 1;
                else hi = mid - 1;
            }
            twin[e] = t;
        }
    }
}

/* The bin whose rotated direction is closest to direction dir:
   argmax_b q_b . dir, ties -> lowest b. */
static int closest_bin(const int32_t *qb, int nbins, const int32_t *dir) {
    int best = 0;
    int64_t bestd = idot(qb, dir);
    for (int b = 1; b < nbins; ++b) {
        int64_t d = idot(qb + 3 * b, dir);
        if (d > bestd) {
            best = b;
            bestd = d;
        }
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* Simulation state                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    int nbins;
    const double *pos;      /* borrowed */
    int64_t *row_ptr;
    int32_t *col;
    uint8_t *flags;
    double *A, *tau_max, *R0;
    int32_t *qedge;
    uint8_t *straight;
    double *mean_len;
    double *bins;
    int nsrc;
    int32_t *src_v;
    double *src_rate;
    double *I, *Inew;       /* incoming photons per vertex per bin */
    double *y;
    double budget[4];       /* emitted, absorbed, escaped, in flight */
    int64_t step;
    uint64_t seed;
    double kappa, fc, tol;
    int max_sub;
    int64_t total_sub, total_capped;
    /* ballistic and combined transport (Sect. 2.2.2, 2.2.4) */
    int transport;
    double tau_switch;
    uint8_t *stb;           /* nnz*4: ballistic straight set of every in-edge */
    int64_t *twin;          /* nnz: index of edge i->k in k's row */
    double *Pb, *Pbn;       /* nnz*nbins: bin packets arrived along each in-edge */
    double *Pe, *Pen;       /* nnz: edge packets arrived along each in-edge */
    double *Ev;             /* nnz: a thick vertex's photons per in-edge */
    double *S;              /* n: a thick source's photons of this step */
    uint8_t *thick;         /* n: the vertex's mode in the current step */
    /* diffuse recombination radiation (Sect. 2.2.1, 4.5) */
    double ground;          /* (alpha_A - alpha_B) / alpha_A */
    double *D;              /* n, or NULL: recombination photons of the last step, emitted next */
    double diffuse_emitted; /* photons emitted by recombining cells so far */
    int threads;            /* > 1: the direction-conserving sweep on that many threads */
} ox_sim;

typedef struct {
    int nbins;
    uint64_t seed;
    double sigma, alpha_B, kappa, chem_frac, chem_tol;
    int chem_max_sub;
    int transport;      /* 0 direction conserving, 1 ballistic, 2 combined */
    double tau_switch;  /* combined: ballistic where y tau_max >= tau_switch */
    double alpha_A;     /* 0: on-the-spot (case B); > 0: case A with the ground-level
                           recombination photons re-emitted */
} ox_params;

ox_sim *ox_create(const ox_params *p, int64_t n, const double *pos, const int64_t *row_ptr,
                  const int32_t *col, const double *nH, const double *vol, const uint8_t *flags,
                  const double *y0, const double *bins) {
    if (p->alpha_A != 0.0 && !(p->alpha_A >= p->alpha_B)) return NULL;
    ox_sim *s = (ox_sim *)calloc(1, sizeof(ox_sim));
    int64_t nnz = row_ptr[n];
    s->n = n;
    s->nbins = p->nbins;
    s->pos = pos;
    s->row_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    memcpy(s->row_ptr, row_ptr, sizeof(int64_t) * (size_t)(n + 1));
    s->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    memcpy(s->col, col, sizeof(int32_t) * (size_t)nnz);
    s->flags = (uint8_t *)malloc((size_t)n + 1);
    memcpy(s->flags, flags, (size_t)n);
    s->bins = (double *)malloc(sizeof(double) * 3 * (size_t)p->nbins);
    memcpy(s->bins, bins, sizeof(double) * 3 * (size_t)p->nbins);
    s->qedge = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(nnz ? nnz : 1));
    s->straight = (uint8_t *)malloc(4 * (size_t)(nnz ? nnz : 1));
    s->mean_len = (double *)malloc(sizeof(double) * (size_t)n);
    ox_edge_tables(n, pos, s->row_ptr, s->col, s->qedge, s->straight, s->mean_len);
    s->kappa = p->kappa > 0.0 ? p->kappa
                              : ox_kappa(n, pos, s->row_ptr, s->col, s->flags, s->qedge,
                                         s->straight, p->nbins, bins);
    s->A = (double *)malloc(sizeof(double) * (size_t)n);
    s->tau_max = (double *)malloc(sizeof(double) * (size_t)n);
    s->R0 = (double *)malloc(sizeof(double) * (size_t)n);
    s->y = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        s->A[i] = nH[i] * vol[i];
        s->tau_max[i] = nH[i] * p->sigma * (s->kappa * s->mean_len[i]);
        s->R0[i] = (p->alpha_A > 0.0 ? p->alpha_A : p->alpha_B) * nH[i];
        s->y[i] = y0 ? y0[i] : 1.0;
    }
    size_t nI = (size_t)n * (size_t)p->nbins;
    s->I = (double *)calloc(nI ? nI : 1, sizeof(double));
    s->Inew = (double *)calloc(nI ? nI : 1, sizeof(double));
    s->seed = p->seed;
    s->fc = p->chem_frac;
    s->tol = p->chem_tol;
    s->max_sub = p->chem_max_sub;
    s->transport = p->transport;
    s->tau_switch = p->tau_switch;
    if (p->alpha_A > 0.0) {
        s->ground = (p->alpha_A - p->alpha_B) / p->alpha_A;
        s->D = (double *)calloc((size_t)n + 1, sizeof(double));
    }
    if (s->transport != 0) {
        size_t m = nnz ? (size_t)nnz : 1;
        s->stb = (uint8_t *)malloc(4 * m);
        s->twin = (int64_t *)malloc(sizeof(int64_t) * m);
        ox_ballistic_tables(n, s->row_ptr, s->col, s->qedge, s->stb, s->twin);
        s->Pb = (double *)calloc(m * (size_t)p->nbins, sizeof(double));
        s->Pbn = (double *)calloc(m * (size_t)p->nbins, sizeof(double));
        s->Pe = (double *)calloc(m, sizeof(double));
        s->Pen = (double *)calloc(m, sizeof(double));
        s->Ev = (double *)calloc(m, sizeof(double));
        s->S = (double *)calloc((size_t)n + 1, sizeof(double));
        s->thick = (uint8_t *)calloc((size_t)n + 1, 1);
    }
    return s;
}

void ox_destroy(ox_sim *s) {
    if (!s) return;
    free(s->row_ptr); free(s->col); free(s->flags); free(s->bins); free(s->qedge);
    free(s->straight); free(s->mean_len); free(s->A); free(s->tau_max); free(s->R0);
    free(s->y); free(s->I); free(s->Inew); free(s->src_v); free(s->src_rate);
    free(s->stb); free(s->twin); free(s->Pb); free(s->Pbn); free(s->Pe); free(s->Pen);
    free(s->Ev); free(s->S); free(s->thick); free(s->D);
    free(s);
}

int ox_add_source(ox_sim *s, int32_t v, double rate) {
    if (v < 0 || v >= s->n) return -1;
    s->src_v = (int32_t *)realloc(s->src_v, sizeof(int32_t) * (size_t)(s->nsrc + 1));
    s->src_rate = (double *)realloc(s->src_rate, sizeof(double) * (size_t)(s->nsrc + 1));
    s->src_v[s->nsrc] = v;
    s->src_rate[s->nsrc] = rate;
    s->nsrc++;
    return 0;
}

/* The interaction and transport of one direction-conserving step on
   s->threads threads, with the results of the serial loop of ox_one_step bit
   for bit (the tests hold it to that).  Only what is independent per vertex
   runs in parallel, and every sum keeps the serial order:
     1. per vertex i (parallel): N_in, the chemistry, and for every bin b the
        transmitted O_i[b] and the straight set S(i, b) it goes to;
     2. the budget (serial, i then b ascending, as the serial loop adds it);
     3. the transport, as its definition reads: I'_j[b] = sum over the
        vertices i with j in S(i, b), in ascending i, of O_i[b] / |S(i, b)|.
        Each j (parallel) walks its own neighbours, which are the only
        candidates and come in ascending order, so every bin adds its terms in
        the order of the serial push. */
static void sweep_threaded(ox_sim *s, double dt, const int32_t *qb) {
    const int nb = s->nbins;
    const int64_t n = s->n;
    const size_t nI = (size_t)n * (size_t)nb;
    double *nin = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *O = (double *)malloc(sizeof(double) * (nI ? nI : 1));       /* O_i[b] */
    int64_t *sset = (int64_t *)malloc(sizeof(int64_t) * (nI ? nI : 1)); /* edge of S(i,b), -1: escapes */
    int *nsub = (int *)calloc((size_t)n + 1, sizeof(int));
    int *capped = (int *)calloc((size_t)n + 1, sizeof(int));
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->threads)
    for (int64_t i = 0; i < n; ++i) {
        const double *Ii = s->I + (size_t)i * nb;
        double N_in = 0.0;
        for (int b = 0; b < nb; ++b) N_in += Ii[b];
        nin[i] = N_in;
        if (s->flags[i] & 1) continue;
        double rec = 0.0;
        double f = ox_chem_rec(&s->y[i], N_in, dt, s->A[i], s->tau_max[i], s->R0[i], s->fc, s->tol,
                               s->max_sub, &nsub[i], &capped[i], &rec);
        if (s->D) s->D[i] = s->ground * (s->A[i] * rec);
        int64_t r0 = s->row_ptr[i], r1 = s->row_ptr[i + 1];
        for (int b = 0; b < nb; ++b) {
            O[(size_t)i * nb + b] = Ii[b] * f;
            int64_t e = -1;
            if (r1 > r0) {
                int k = associate(qb + 3 * b, s->qedge, r0, r1);
                if (s->straight[4 * (r0 + k) + 3] > 0) e = r0 + k;
            }
            sset[(size_t)i * nb + b] = e;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        s->total_sub += nsub[i];
        s->total_capped += capped[i];
        if (s->flags[i] & 1) {
            s->budget[2] += nin[i];
            continue;
        }
        double out_sum = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double Ob = O[(size_t)i * nb + b];
            out_sum += Ob;
            if (sset[(size_t)i * nb + b] < 0) s->budget[2] += Ob;
        }
        s->budget[1] += nin[i] - out_sum;
    }
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->threads)
    for (int64_t j = 0; j < n; ++j) {
        double *Ij = s->Inew + (size_t)j * nb;
        for (int b = 0; b < nb; ++b) Ij[b] = 0.0;
        for (int64_t ej = s->row_ptr[j]; ej < s->row_ptr[j + 1]; ++ej) {
            const int64_t i = s->col[ej];
            if (s->flags[i] & 1) continue;  /* a sink sends nothing */
            const int64_t r0 = s->row_ptr[i];
            for (int b = 0; b < nb; ++b) {
                const int64_t e = sset[(size_t)i * nb + b];
                if (e < 0) continue;
                const uint8_t *st = s->straight + 4 * e;
                const int cnt = st[3];
                for (int m = 0; m < cnt; ++m) {
                    if (s->col[r0 + st[m]] == j) {
                        Ij[b] += O[(size_t)i * nb + b] / cnt;
                        break;
                    }
                }
            }
        }
    }
    free(nin); free(O); free(sset); free(nsub); free(capped);
    double *t = s->I;
    s->I = s->Inew;
    s->Inew = t;
    double inflight = 0.0;
    for (size_t e = 0; e < nI; ++e) inflight += s->I[e];
    s->budget[3] = inflight;
    s->step++;
}

/* One radiative-transfer step of length dt (Sect. 4.6). */
static void ox_one_step(ox_sim *s, double dt) {
    const int nb = s->nbins;
    const int64_t n = s->n;
    double R[9];
    ox_rotation(s->seed, s->step, R);
    int32_t *qb = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)nb);
    ox_rotated_bins(R, nb, s->bins, qb);

    /* photons in flight were binned in the previous step's orientation:
       move every packet to the closest bin of this step's orientation */
    if (s->step > 0) {
        double Rp[9];
        ox_rotation(s->seed, s->step - 1, Rp);
        int32_t *qp = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)nb);
        int32_t *map = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
        double *tmp = (double *)malloc(sizeof(double) * (size_t)nb);
        ox_rotated_bins(Rp, nb, s->bins, qp);
        ox_bin_map(nb, qp, qb, map);
        if (s->threads > 1) {  /* the same loop, vertices split over threads */
#pragma omp parallel num_threads(s->threads)
            {
                double *t = (double *)malloc(sizeof(double) * (size_t)nb);
#pragma omp for schedule(static)
                for (int64_t i = 0; i < n; ++i) {
                    double *Ii = s->I + (size_t)i * nb;
                    for (int b = 0; b < nb; ++b) t[b] = 0.0;
                    for (int b = 0; b < nb; ++b) t[map[b]] += Ii[b];
                    for (int b = 0; b < nb; ++b) Ii[b] = t[b];
                }
                free(t);
            }
        } else {
            for (int64_t i = 0; i < n; ++i) {
                double *Ii = s->I + (size_t)i * nb;
                for (int b = 0; b < nb; ++b) tmp[b] = 0.0;
                for (int b = 0; b < nb; ++b) tmp[map[b]] += Ii[b];
                for (int b = 0; b < nb; ++b) Ii[b] = tmp[b];
            }
        }
        free(qp); free(map); free(tmp);
    }

    /* sources: an equal share of the step's photons in every bin */
    for (int k = 0; k < s->nsrc; ++k) {
        double Nstep = s->src_rate[k] * dt;
        double share = Nstep / nb;
        double *Iv = s->I + (size_t)s->src_v[k] * nb;
        for (int b = 0; b < nb; ++b) Iv[b] += share;
        s->budget[0] += Nstep;
    }

    /* diffuse radiation: every cell emits the ground-level recombination
       photons of the last step like a source, an equal share in every bin */
    if (s->D) {
        for (int64_t i = 0; i < n; ++i) {
            if (!(s->D[i] > 0.0)) continue;
            double share = s->D[i] / nb;
            double *Iv = s->I + (size_t)i * nb;
            for (int b = 0; b < nb; ++b) Iv[b] += share;
            s->budget[0] += s->D[i];
            s->diffuse_emitted += s->D[i];
            s->D[i] = 0.0;
        }
    }

    if (s->threads > 1) {
        sweep_threaded(s, dt, qb);
        free(qb);
        return;
    }
    memset(s->Inew, 0, sizeof(double) * (size_t)n * nb);
    for (int64_t i = 0; i < n; ++i) {
        double *Ii = s->I + (size_t)i * nb;
        double N_in = 0.0;
        for (int b = 0; b < nb; ++b) N_in += Ii[b];
        if (s->flags[i] & 1) {           /* sink: leaves the volume */
            s->budget[2] += N_in;
            continue;
        }
        int nsub = 0, capped = 0;
        double rec = 0.0;
        double f = ox_chem_rec(&s->y[i], N_in, dt, s->A[i], s->tau_max[i], s->R0[i], s->fc, s->tol,
                               s->max_sub, &nsub, &capped, &rec);
        s->total_sub += nsub;
        s->total_capped += capped;
        if (s->D) s->D[i] = s->ground * (s->A[i] * rec);
        int64_t r0 = s->row_ptr[i], r1 = s->row_ptr[i + 1];
        double out_sum = 0.0;
        for (int b = 0; b < nb; ++b) {
            double O = Ii[b] * f;
            out_sum += O;
            if (r1 == r0) {
                s->budget[2] += O;
                continue;
            }
            int k = associate(qb + 3 * b, s->qedge, r0, r1);
            const uint8_t *st = s->straight + 4 * (r0 + k);
            int cnt = st[3];
            if (cnt == 0) {
                s->budget[2] += O;
                continue;
            }
            double w = O / cnt;
            for (int m = 0; m < cnt; ++m) s->Inew[(size_t)s->col[r0 + st[m]] * nb + b] += w;
        }
        s->budget[1] += N_in - out_sum;
    }
    double *t = s->I;
    s->I = s->Inew;
    s->Inew = t;
    double inflight = 0.0;
    for (size_t e = 0; e < (size_t)n * nb; ++e) inflight += s->I[e];
    s->budget[3] = inflight;
    s->step++;
    free(qb);
}

/* One step of ballistic or combined transport (Sect. 2.2.2, 2.2.4).
   A vertex is thick (ballistic) in a step when its optical depth y tau_max
   reaches tau_switch (always, in ballistic transport), else thin (direction
   conserving); sinks keep bins.  Photons arrive along in-edges and are kept
   as the receiver's mode keeps them: a thin vertex in direction bins (bin
   packets go to the closest bin of this step's orientation, edge packets to
   the bin closest to the direction they travelled), a thick vertex per
   in-edge.  A thin vertex sends its bins as in ox_one_step; a thick vertex
   sends the photons of each in-edge to that edge's ballistic straight set,
   and a thick source (or a thick cell re-emitting recombination photons)
   its own photons to all neighbours in equal parts (Sect. 2.2.1). */
static void ox_one_step_ballistic(ox_sim *s, double dt) {
    const int nb = s->nbins;
    const int64_t n = s->n;
    const int64_t nnz = s->row_ptr[n];
    double R[9];
    ox_rotation(s->seed, s->step, R);
    int32_t *qb = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)nb);
    int32_t *map = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)nb);
    ox_rotated_bins(R, nb, s->bins, qb);
    if (s->step > 0) {
        double Rp[9];
        ox_rotation(s->seed, s->step - 1, Rp);
        int32_t *qp = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)nb);
        ox_rotated_bins(Rp, nb, s->bins, qp);
        ox_bin_map(nb, qp, qb, map);
        free(qp);
    } else {
        for (int b = 0; b < nb; ++b) map[b] = b;
    }

    /* the mode of every vertex in this step */
    for (int64_t i = 0; i < n; ++i)
        s->thick[i] = !(s->flags[i] & 1) &&
                      (s->transport == 1 || s->y[i] * s->tau_max[i] >= s->tau_switch);

    /* arrivals */
    for (int64_t i = 0; i < n; ++i) {
        int64_t r0 = s->row_ptr[i], r1 = s->row_ptr[i + 1];
        double *Ii = s->I + (size_t)i * nb;
        for (int b = 0; b < nb; ++b) Ii[b] = 0.0;
        s->S[i] = 0.0;
        if (!s->thick[i]) {
            for (int b = 0; b < nb; ++b) tmp[b] = 0.0;
            for (int64_t e = r0; e < r1; ++e)
                for (int b = 0; b < nb; ++b) tmp[b] += s->Pb[(size_t)e * nb + b];
            for (int b = 0; b < nb; ++b) Ii[map[b]] += tmp[b];
            for (int64_t e = r0; e < r1; ++e) {
                if (s->Pe[e] == 0.0) continue;
                int32_t dir[3] = {-s->qedge[3 * e], -s->qedge[3 * e + 1], -s->qedge[3 * e + 2]};
                Ii[closest_bin(qb, nb, dir)] += s->Pe[e];
            }
        } else {
            for (int64_t e = r0; e < r1; ++e) {
                double a = 0.0;
                for (int b = 0; b < nb; ++b) a += s->Pb[(size_t)e * nb + b];
                s->Ev[e] = a + s->Pe[e];
            }
        }
    }

    /* sources: in bins at a thin vertex, the vertex's own photons at a thick one */
    for (int k = 0; k < s->nsrc; ++k) {
        int64_t v = s->src_v[k];
        double Nstep = s->src_rate[k] * dt;
        s->budget[0] += Nstep;
        if (s->thick[v]) {
            s->S[v] += Nstep;
        } else {
            double share = Nstep / nb;
            double *Iv = s->I + (size_t)v * nb;
            for (int b = 0; b < nb; ++b) Iv[b] += share;
        }
    }

    /* diffuse radiation: the ground-level recombination photons of the last
       step, emitted like a source's */
    if (s->D) {
        for (int64_t i = 0; i < n; ++i) {
            if (!(s->D[i] > 0.0)) continue;
            if (s->thick[i]) {
                s->S[i] += s->D[i];
            } else {
                double share = s->D[i] / nb;
                double *Iv = s->I + (size_t)i * nb;
                for (int b = 0; b < nb; ++b) Iv[b] += share;
            }
            s->budget[0] += s->D[i];
            s->diffuse_emitted += s->D[i];
            s->D[i] = 0.0;
        }
    }

    /* interaction and transport */
    memset(s->Pbn, 0, sizeof(double) * (size_t)(nnz ? nnz : 1) * nb);
    memset(s->Pen, 0, sizeof(double) * (size_t)(nnz ? nnz : 1));
    for (int64_t i = 0; i < n; ++i) {
        int64_t r0 = s->row_ptr[i], r1 = s->row_ptr[i + 1];
        const double *Ii = s->I + (size_t)i * nb;
        double N_in = 0.0;
        if (s->thick[i]) {
            for (int64_t e = r0; e < r1; ++e) N_in += s->Ev[e];
            N_in += s->S[i];
        } else {
            for (int b = 0; b < nb; ++b) N_in += Ii[b];
        }
        if (s->flags[i] & 1) {
            s->budget[2] += N_in;
            continue;
        }
        int nsub = 0, capped = 0;
        double rec = 0.0;
        double f = ox_chem_rec(&s->y[i], N_in, dt, s->A[i], s->tau_max[i], s->R0[i], s->fc, s->tol,
                               s->max_sub, &nsub, &capped, &rec);
        s->total_sub += nsub;
        s->total_capped += capped;
        if (s->D) s->D[i] = s->ground * (s->A[i] * rec);
        double out_sum = 0.0;
        if (!s->thick[i]) {
            for (int b = 0; b < nb; ++b) {
                double O = Ii[b] * f;
                out_sum += O;
                if (r1 == r0) {
                    s->budget[2] += O;
                    continue;
                }
                int k = associate(qb + 3 * b, s->qedge, r0, r1);
                const uint8_t *st = s->straight + 4 * (r0 + k);
                int cnt = st[3];
                if (cnt == 0) {
                    s->budget[2] += O;
                    continue;
                }
                double w = O / cnt;
                for (int m = 0; m < cnt; ++m) s->Pbn[(size_t)s->twin[r0 + st[m]] * nb + b] += w;
            }
        } else {
            for (int64_t e = r0; e < r1; ++e) {
                double O = s->Ev[e] * f;
                out_sum += O;
                const uint8_t *st = s->stb + 4 * e;
                int cnt = st[3];
                if (cnt == 0) {
                    s->budget[2] += O;
                    continue;
                }
                double w = O / cnt;
                for (int m = 0; m < cnt; ++m) s->Pen[s->twin[r0 + st[m]]] += w;
            }
            if (s->S[i] != 0.0) {
                double O = s->S[i] * f;
                out_sum += O;
                if (r1 == r0) {
                    s->budget[2] += O;
                } else {
                    double w = O / (double)(r1 - r0);
                    for (int64_t e = r0; e < r1; ++e) s->Pen[s->twin[e]] += w;
                }
            }
        }
        s->budget[1] += N_in - out_sum;
    }
    double *t = s->Pb;
    s->Pb = s->Pbn;
    s->Pbn = t;
    t = s->Pe;
    s->Pe = s->Pen;
    s->Pen = t;
    double inflight = 0.0;
    for (size_t e = 0; e < (size_t)nnz * nb; ++e) inflight += s->Pb[e];
    for (int64_t e = 0; e < nnz; ++e) inflight += s->Pe[e];
    s->budget[3] = inflight;
    s->step++;
    free(qb);
    free(map);
    free(tmp);
}

/* Threads of the direction-conserving sweep (1: the serial loop). */
void ox_set_threads(ox_sim *s, int threads) { s->threads = threads > 1 ? threads : 1; }

void ox_step(ox_sim *s, double dt, int nsteps) {
    for (int k = 0; k < nsteps; ++k) {
        if (s->transport == 0) ox_one_step(s, dt);
        else ox_one_step_ballistic(s, dt);
    }
}

/* Photons in flight towards every vertex (the packets on its in-edges). */
void ox_get_inflight(const ox_sim *s, double *out) {
    const int nb = s->nbins;
    for (int64_t i = 0; i < s->n; ++i) {
        double a = 0.0;
        if (s->transport == 0) {
            for (int b = 0; b < nb; ++b) a += s->I[(size_t)i * nb + b];
        } else {
            for (int64_t e = s->row_ptr[i]; e < s->row_ptr[i + 1]; ++e) {
                for (int b = 0; b < nb; ++b) a += s->Pb[(size_t)e * nb + b];
                a += s->Pe[e];
            }
        }
        out[i] = a;
    }
}

/* The ballistic tables and the modes of the last step (1 = thick). */
void ox_get_ballistic(const ox_sim *s, uint8_t *stb, int64_t *twin, uint8_t *thick) {
    int64_t nnz = s->row_ptr[s->n];
    if (s->transport == 0) return;
    memcpy(stb, s->stb, 4 * (size_t)nnz);
    memcpy(twin, s->twin, sizeof(int64_t) * (size_t)nnz);
    memcpy(thick, s->thick, (size_t)s->n);
}

void ox_get_y(const ox_sim *s, double *out) { memcpy(out, s->y, sizeof(double) * (size_t)s->n); }
void ox_set_y(ox_sim *s, const double *in) { memcpy(s->y, in, sizeof(double) * (size_t)s->n); }
void ox_get_I(const ox_sim *s, double *out) {
    memcpy(out, s->I, sizeof(double) * (size_t)s->n * s->nbins);
}
void ox_set_I(ox_sim *s, const double *in) {
    memcpy(s->I, in, sizeof(double) * (size_t)s->n * s->nbins);
}
void ox_get_budget(const ox_sim *s, double *out) { memcpy(out, s->budget, sizeof(double) * 4); }
double ox_get_kappa(const ox_sim *s) { return s->kappa; }
int64_t ox_get_step(const ox_sim *s) { return s->step; }
void ox_get_stats(const ox_sim *s, int64_t *out) {
    out[0] = s->total_sub;
    out[1] = s->total_capped;
}
void ox_get_vertex_consts(const ox_sim *s, double *A, double *tau_max, double *R0) {
    memcpy(A, s->A, sizeof(double) * (size_t)s->n);
    memcpy(tau_max, s->tau_max, sizeof(double) * (size_t)s->n);
    memcpy(R0, s->R0, sizeof(double) * (size_t)s->n);
}
void ox_get_tables(const ox_sim *s, int32_t *qedge, uint8_t *straight, double *mean_len) {
    int64_t nnz = s->row_ptr[s->n];
    memcpy(qedge, s->qedge, sizeof(int32_t) * 3 * (size_t)nnz);
    memcpy(straight, s->straight, 4 * (size_t)nnz);
    memcpy(mean_len, s->mean_len, sizeof(double) * (size_t)s->n);
}
/* association of every (vertex, bin) for the rotation of step `step` */
void ox_associate_all(const ox_sim *s, int64_t step, int32_t *assoc /* n*nbins */) {
    double R[9];
    ox_rotation(s->seed, step, R);
    int32_t *qb = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)s->nbins);
    ox_rotated_bins(R, s->nbins, s->bins, qb);
    for (int64_t i = 0; i < s->n; ++i)
        for (int b = 0; b < s->nbins; ++b)
            assoc[(size_t)i * s->nbins + b] =
                (s->row_ptr[i + 1] > s->row_ptr[i])
                    ? associate(qb + 3 * b, s->qedge, s->row_ptr[i], s->row_ptr[i + 1])
                    : -1;
    free(qb);
}

/* ------------------------------------------------------------------------ */
/* Dynamic grid (Sect. 2.1.4): vertices where the optical depth fell are     */
/* removed, but not below a minimum resolution.                              */
/*   candidate: not a sink, not a source, neutral fraction y < y_thresh (the */
/*   cell became transparent) and local spacing (mean edge length) below     */
/*   min_spacing (finer than the minimum resolution);                        */
/*   removed: a candidate all of whose candidate neighbours have larger ids  */
/*   (no two removed vertices are adjacent).                                 */
/* Returns the number removed; their ids, ascending, in removed_out.         */
/* ------------------------------------------------------------------------ */
int64_t ox_mark_removal(const ox_sim *s, double y_thresh, double min_spacing,
                        int32_t *removed_out) {
    const int64_t n = s->n;
    uint8_t *cand = (uint8_t *)calloc((size_t)n + 1, 1);
    for (int64_t i = 0; i < n; ++i) {
        int is_src = 0;
        for (int k = 0; k < s->nsrc; ++k) is_src |= (s->src_v[k] == i);
        cand[i] = !(s->flags[i] & 1) && !is_src && s->y[i] < y_thresh && s->mean_len[i] < min_spacing;
    }
    int64_t nr = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!cand[i]) continue;
        int ok = 1;
        for (int64_t e = s->row_ptr[i]; e < s->row_ptr[i + 1]; ++e) {
            int64_t j = s->col[e];
            if (cand[j] && j < i) ok = 0;
        }
        if (ok) removed_out[nr++] = (int32_t)i;
    }
    free(cand);
    return nr;
}

/* Photons arriving at a removed vertex go to its nearest surviving neighbour,
   bin by bin (ties -> lowest id), removed vertices in ascending order.
   I is n x nbins (the state between steps). */
void ox_hand_over(const ox_sim *s, int64_t nr, const int32_t *removed, double *I) {
    uint8_t *rem = (uint8_t *)calloc((size_t)s->n + 1, 1);
    for (int64_t k = 0; k < nr; ++k) rem[removed[k]] = 1;
    for (int64_t k = 0; k < nr; ++k) {
        int64_t r = removed[k];
        int64_t best = -1;
        double bestd = 0.0;
        for (int64_t e = s->row_ptr[r]; e < s->row_ptr[r + 1]; ++e) {
            int64_t j = s->col[e];
            if (rem[j]) continue;
            double dx = s->pos[3 * j] - s->pos[3 * r], dy = s->pos[3 * j + 1] - s->pos[3 * r + 1],
                   dz = s->pos[3 * j + 2] - s->pos[3 * r + 2];
            double d2 = (dx * dx + dy * dy) + dz * dz;
            if (best < 0 || d2 < bestd || (d2 == bestd && j < best)) {
                best = j;
                bestd = d2;
            }
        }
        if (best < 0) continue;
        for (int b = 0; b < s->nbins; ++b) I[(size_t)best * s->nbins + b] += I[(size_t)r * s->nbins + b];
    }
    free(rem);
}

void ox_set_step(ox_sim *s, int64_t step) { s->step = step; }

/* Diffuse radiation: each cell's photons waiting for the next step (zeros
   without diffuse radiation) and the photons recombining cells emitted. */
double ox_get_diffuse(const ox_sim *s, double *pending) {
    for (int64_t i = 0; i < s->n; ++i) pending[i] = s->D ? s->D[i] : 0.0;
    return s->diffuse_emitted;
}
void ox_set_budget(ox_sim *s, const double *b) { memcpy(s->budget, b, sizeof(double) * 4); }
