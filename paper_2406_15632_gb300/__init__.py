"""qmcrt: quasi-Monte Carlo radiative transfer on GB300 (sm_103a)."""
