"""Plain, slow, CPU FP64 oracle for the nested-dissection selected-inversion density path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
leg may import anything here; the library never does.  It shares no code with the CUDA path.

Modules (each cites the passage of the paper it follows):
  poles        - continued-fraction poles/residues of Eq. (7) and the pole-form Fermi function
  dense        - rho by the generalized eigenproblem (Eqs. 2, 5) and by Eq. (8); G by Eq. (6);
                 energy density matrix (Eq. 10); density of states (Eq. 41)
  closed_form  - the open s-valent chain spectrum (a pin for `dense`)
  nd           - geometric nested dissection, Sec. II.C.1 steps (i)-(v), and symbolic fill
  recurrence   - the paper's recurrence formulas, Eqs. (28)-(32) and (38)-(39), on App. A
  eigen        - selected eigenstates near an energy (App. B): definition, three-step solve
                 (B8)-(B15) and the block shift-invert iteration (B2)-(B3)
  mlp          - FP64 forward/backward of the chemical-potential seed network
"""
