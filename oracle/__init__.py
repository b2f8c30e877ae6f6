"""CPU FP64 oracle for the walk-based Laplacians (test infrastructure only).

Only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` /
`--impl reference` legs of `bench.py` may import or execute anything in this
package. The CUDA library never calls it and shares no code with it; the two
meet only in the seeded input generators of `wlgen`.

Everything here is plain, dense and slow on purpose: each function follows a
definition of the paper (Arrigo and Durastante, "Walk based Laplacians for
Modeling Diffusion on Complex Networks") and cites the section, equation or
proposition it restates. Library primitives (matrix products, dense solves,
symmetric eigendecompositions) serve as single steps; nothing is blocked,
fused or reordered beyond the definition.

Modules
  graph      dense adjacency, degrees (Sec. 2)
  walks      q_k recurrences, f(A) and phi(A, c) two independent ways,
             walk degrees, Laplacian, its action, diffusion (Sec. 3)
  spectral   companion matrix Z (Eq. Zdef), rho(Z), lambda_max(A)
  brute      brute-force (weighted) walk enumeration (Sec. 3.2)
  xnys       exact trace and the literal leave-one-out XNysTrace (Alg. 1)
  philox     Philox4x32-10 counter-based generator and Box-Muller normals
  mlp        FP64 forward / backward / Adam for the warm-start network
  features   local node features for the warm-start network
"""
