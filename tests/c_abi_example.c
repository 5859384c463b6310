/* A plain C (C99) user of include/mera.h: the critical Ising chain on blocked
 * spin pairs (d_b = 4), a binary MERA with chi = 4 and two transition layers,
 * a seeded random start (mera_init_random), 50 L-BFGS iterations through
 * mera_solve, the gradient copied to host memory.  Built by
 * tests/test_c_abi.py (compile and link on any machine; run on a GPU).
 * Prints "energy_per_spin <e> gnorm <g> iters <n>" and exits 0. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "mera.h"

/* Pauli matrices as 2 x 2 row-major arrays */
static const double PX[4] = {0, 1, 1, 0};
static const double PZ[4] = {1, 0, 0, -1};
static const double ID[4] = {1, 0, 0, 1};

/* c (n1 n2 x n1 n2) = a (n1 x n1) kron b (n2 x n2) */
static void kron(const double* a, int n1, const double* b, int n2, double* c) {
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n1; ++j)
            for (int k = 0; k < n2; ++k)
                for (int l = 0; l < n2; ++l)
                    c[(i * n2 + k) * (n1 * n2) + j * n2 + l] = a[i * n1 + j] * b[k * n2 + l];
}

int main(void) {
    /* bond term on spins: -X X - (Z 1 + 1 Z) / 2 */
    double xx[16], z1[16], iz[16], bond[16];
    kron(PX, 2, PX, 2, xx);
    kron(PZ, 2, ID, 2, z1);
    kron(ID, 2, PZ, 2, iz);
    for (int i = 0; i < 16; ++i) bond[i] = -xx[i] - 0.5 * (z1[i] + iz[i]);
    /* blocked two-site term hb = (bond x 1 + 1 x bond) / 2 + 1 x bond x 1, then
       the three-site term h3 = (hb x 1 + 1 x hb) / 2 (sites of dimension 4) */
    double id4[16] = {0}, id2[4] = {1, 0, 0, 1};
    for (int i = 0; i < 4; ++i) id4[i * 5] = 1.0;
    double a[256], b[256], t[64], inter[256], hb[256];
    kron(bond, 4, id4, 4, a);
    kron(id4, 4, bond, 4, b);
    kron(id2, 2, bond, 4, t);
    kron(t, 8, id2, 2, inter);
    for (int i = 0; i < 256; ++i) hb[i] = 0.5 * (a[i] + b[i]) + inter[i];
    static double h3[4096], p[4096], q[4096];
    kron(hb, 16, id4, 4, p);
    kron(id4, 4, hb, 16, q);
    for (int i = 0; i < 4096; ++i) h3[i] = 0.5 * (p[i] + q[i]);

    mera_config cfg;
    mera_config_default(&cfg, 4, 4, 2);
    mera_t m = NULL;
    int rc = mera_create(&cfg, h3, NULL, &m);
    if (rc != MERA_OK) {
        fprintf(stderr, "mera_create: %s\n", mera_strerror(rc));
        return 1;
    }
    rc = mera_init_random(m, 7);
    mera_solve_opts opts = {0, 50, 1e-10};
    mera_solve_result res;
    if (rc == MERA_OK) rc = mera_solve(m, &opts, &res);
    if (rc != MERA_OK) {
        fprintf(stderr, "%s: %s\n", mera_strerror(rc), mera_last_error(m));
        mera_destroy(m);
        return 1;
    }
    /* the gradient in host memory, one array per tensor */
    int nt = mera_num_tensors(m);
    void* grads[16];
    for (int i = 0; i < nt; ++i) {
        int64_t r, c;
        mera_tensor_shape(m, i, &r, &c);
        grads[i] = malloc(sizeof(double) * (size_t)(r * c));
    }
    double e = 0.0;
    rc = mera_energy_grad(m, &e, grads, NULL);
    for (int i = 0; i < nt; ++i) free(grads[i]);
    mera_destroy(m);
    if (rc != MERA_OK || !isfinite(e)) return 1;
    printf("energy_per_spin %.12f gnorm %.3e iters %d\n", e / 2, res.gnorm, res.iters);
    return 0;
}
