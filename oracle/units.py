"""Atomic units (hbar = m_e = e = 1). Test infrastructure only.

The paper's inputs are in Angstrom / eV / amu (Table 1); this project's workloads
are already in bohr, eV and amu, so only energies and masses are converted.
"""
HARTREE_IN_EV = 27.211386245988
EV = 1.0 / HARTREE_IN_EV          # hartree per eV
AMU = 1822.888486                 # electron masses per unified atomic mass unit
