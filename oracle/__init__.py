"""FP64 CPU oracle for the depth-pruned message-passing potential.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library; both receive the same seeded inputs from the
``synth`` module.

Modules
  neighbors  periodic minimum-image edge sets: O(N^2) brute force (the
             definition) and a plain cell list (checked against it).
  model      the network in float64 torch with autograd forces F = -dE/dr.
  partition  spatial-grid root sets, geometric and K-hop BFS halos and the
             partitioned evaluation with root-only seeding.
  md         velocity-Verlet NVE integration and its energy ledger.
  head       the per-atom correction head, its losses and gradients.
  diag       layer diagnostics (mean feature shift, linear CKA).

Paper anchors (arXiv 2509.21694): the method prunes a message-passing
backbone to its first K layers (Methods, "Message Passing Depth Pruning"),
partitions the atom graph into root sets on a spatial grid and extends each
by a K-hop BFS (Methods, "Graph Partitioning", Stage 1 and Stage 2), and
assembles E as the sum of root energies and F as the sum over partitions of
the gradients of root energies (Methods, "Global Output Integration").  The
paper gives no network equations; the concrete network here is the reading
recorded in the design notes (Bessel basis, polynomial envelope, real
spherical harmonics, radial MLP, receiver sums, per-l node updates).

Parity status per function is stated in each module header.
"""
