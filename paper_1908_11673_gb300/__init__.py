"""GB300-native (sm_103a) Wilson-clover Dirac operator with SU(3) x U(1) links,
C* boundaries and its solvers, behind the C ABI of libqxd (include/qxd.h)."""
