"""CPU FP64 oracle for one damped Gauss-Newton step of the self-similar profile fit.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only the tests, `__graft_entry__.smoke()` and the `cpu_baseline` /
`--impl reference` legs of `bench.py` use it.  It shares no code with the CUDA
library (no kernels, headers, helpers or constant tables); the only module
both sides consume is the seeded input generator, which holds none of the
method's arithmetic.

What it computes (citations are to the paper's Methods section):
  * jets.py     second-order y-jets through arbitrary expressions (plain
                forward-mode calculus; used for the field derivatives the
                residuals need).
  * problems.py the self-similar ansatz (Eq. self-similar), the compactified
                inputs q, beta (Solution Modeling), the symmetry/decay
                envelopes (Eq. ansatz_vorticity and its generalisation), the
                tanh MLP, and the residual operators R_k of each equation.
  * hilbert.py  the discrete Hilbert operator that defines the CCF velocity.
  * gn.py       weighted rows r~, the Jacobian J~ by complex-step
                differentiation (one column per parameter and one for
                lambda), Gram G = J~^T J~, gradient g = J~^T r~, textbook
                Cholesky, damped solve, Armijo line search and the
                Levenberg-Marquardt damping update (Second-order Optimizer).

Pins (each checked by a `-m "not gpu"` test against something other than the
oracle itself): complex-step vs central differences, jet derivatives vs
complex-step in y, residual operators vs a symbolic reduction of each PDE
under the self-similar ansatz, the Boussinesq lambda-inference rule printed in
the paper, Burgers closed-form profiles (residual zero to rounding), Hilbert
transform pairs, odd/even symmetry of every residual, Cholesky vs a library
factorisation, and one GN step on a linear least-squares problem vs the
normal-equations solution.

Parity unpinned: the CCF, IPM and Boussinesq residuals as *physics* (the paper
defers their exact definitions to its Supplementary Information); what is
pinned is the reduction of the standard PDEs under the paper's ansatz.
"""
