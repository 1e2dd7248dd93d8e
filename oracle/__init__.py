"""FP64 CPU oracle for one GNN-MPC real-time-iteration step.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports or calls it, and it imports nothing from the product path.  It shares
no code with the CUDA side: its only common dependency is the seeded input
generator in ``synth``, which holds none of the method's arithmetic.

Everything here is plain numpy in float64, written for readability, not
speed:

* ``gnn``       the GNN dynamics (Sec. V-A, Eq. forward_dynamics) and its exact
                Jacobians by forward-mode chain rule (Eq. linearized_dynamics);
* ``condense``  textbook dense condensing (Eq. condensed_matrices) and the
                paper's per-node recursion (Thm. 1 proof: Eq. sparse_gamma_i_xb,
                Eq. sparse_gamma_i_u, Eq. H, Eq. g, stacked constraints);
* ``qp``        the condensed QP: exact optimum (primal-dual interior point,
                then an equality-constrained solve on the identified active
                set), the ADMM recurrence, KKT certificates, brute force over
                active sets and the uncondensed (x, u) QP for tiny cases;
* ``rti``       one iteration of Algorithm 1 assembled from the above;
* ``warmstart`` the learned ADMM warm start (an addition, not in the paper):
                pooled GNN-latent features, the MLP, its loss gradient and
                the Adam step.

Pins (tests marked ``not gpu``): central finite differences, closed forms for
identity-activation GNNs, the N=1 worked case of the Thm. 1 proof, recursion
versus textbook condensing, the condensed cost versus a direct simulation of
the linear system, the condensed QP versus the uncondensed QP, brute-force
active sets, KKT certificates and Thm. 1's linear flop count; for the warm
start, finite differences of the loss, the linear regime of the MLP, the first
Adam step's sign property and pooling invariances.
"""
