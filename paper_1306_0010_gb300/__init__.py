"""GB300-native gray M1 radiation subcycle (Skinner & Ostriker 2013) behind a C-ABI library."""
