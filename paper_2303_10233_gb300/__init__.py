"""GB300-native enriched Taylor--Hood (Q2--Q1*) Stokes/Oseen Krylov solvers."""
